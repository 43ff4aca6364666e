"""Stored tables and surrogates (Sec. 3.1.1, 3.2.3: tables computed once and kept): a loaded object
reproduces the saved one bit for bit, and a damaged file is refused."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_09568_gb300 as msasm  # noqa: E402
from paper_2107_09568_gb300._lib import EIO, MsasmError  # noqa: E402


@pytest.mark.parametrize("q", [3, (2, 3, 1)])
def test_tables_round_trip_is_bit_exact(tmp_path, q):
    tab = msasm.Tables(synth.micro_cross(3, 0.27), q)
    path = tmp_path / "cross.msasm"
    tab.save(path)
    back = msasm.Tables.load_file(path)
    assert (back.n_T, back.n_nz, back.n_pi, back.qd) == (tab.n_T, tab.n_nz, tab.n_pi, tab.qd)
    assert np.array_equal(back.pairs(), tab.pairs())
    assert torch.equal(back.table(), tab.table())
    for a, b in zip(back.load_table(), tab.load_table()):
        assert torch.equal(a, b)
    for f in range(6):
        assert torch.equal(back.face_table(f), tab.face_table(f))
    # the loaded tables assemble the same matrix, in the FP64 and the FP64-accurate forms
    m = synth.macro_perturbed_cube(seed=3)
    ctrl = torch.tensor(m.ctrl, device="cuda")
    p0, p1 = msasm.Plan(tab, m), msasm.Plan(back, m)
    for prec in ("f64", "f64_emu"):
        assert torch.equal(p1.assemble(ctrl, 1.0, 0.3, prec), p0.assemble(ctrl, 1.0, 0.3, prec)), prec


def test_damaged_table_file_is_refused(tmp_path):
    tab = msasm.Tables(synth.micro_cross(2, 0.3), 2)
    path = tmp_path / "t.msasm"
    tab.save(path)
    raw = bytearray(path.read_bytes())
    flipped = tmp_path / "flipped.msasm"
    raw2 = bytearray(raw)
    raw2[len(raw2) // 2] ^= 0x40                        # one bit inside the FP64 table
    flipped.write_bytes(bytes(raw2))
    with pytest.raises(MsasmError) as e:
        msasm.Tables.load_file(flipped)
    assert e.value.status == EIO and "checksum" in str(e.value)
    short = tmp_path / "short.msasm"
    short.write_bytes(bytes(raw[:-9]))
    with pytest.raises(MsasmError) as e:
        msasm.Tables.load_file(short)
    assert e.value.status == EIO
    # the object that was saved is untouched and still loads
    assert torch.equal(msasm.Tables.load_file(path).table(), tab.table())


def test_surrogate_round_trip_predicts_assembles_and_trains_alike(tmp_path):
    m = synth.macro_quarter_arc(4, 2, 2)
    ctrl = torch.tensor(m.ctrl, device="cuda")
    base = msasm.Tables(synth.micro_cross(3, 0.3), 3)
    plan = msasm.Plan(base, m)
    coef = plan.pullback(ctrl)
    w_train = np.linspace(0.15, 0.40, 8)
    sur = msasm.Surrogate([msasm.Tables(synth.micro_cross(3, w), 3) for w in w_train], w_train, coef,
                          rank=8, hidden=32, power_iters=1, seed=4)
    sur.train(300, 1e-3)
    path = tmp_path / "sur.msasm"
    sur.save(path)
    back = msasm.Surrogate.load_file(path)
    assert (back.rank, back.K, back.n_nz) == (sur.rank, sur.K, sur.n_nz)
    assert torch.equal(back.basis(), sur.basis())
    dw = torch.tensor(synth.width_field(m.n_elem, seed=1), device="cuda")
    assert torch.equal(back.predict(dw), sur.predict(dw))
    assert torch.equal(back.assemble(plan, ctrl, dw), sur.assemble(plan, ctrl, dw))
    # Adam moments and step were stored: training continues identically.  The weights' updates are
    # deterministic; the reported loss is a sum of per-warp partials added atomically, so its last
    # bits depend on the order of those additions.
    h0, h1 = sur.train(50, 1e-3), back.train(50, 1e-3)
    assert np.allclose(h0, h1, rtol=1e-5, atol=0.0)
    assert torch.equal(back.predict(dw), sur.predict(dw))
    # a table file is not a surrogate file
    tpath = tmp_path / "tab.msasm"
    base.save(tpath)
    with pytest.raises(MsasmError) as e:
        msasm.Surrogate.load_file(tpath)
    assert e.value.status == EIO
