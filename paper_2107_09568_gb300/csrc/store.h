// Files of precomputed lookup data (host side).  A file is
//
//   8-byte kind tag | uint32 format version | uint32 byte-order mark 0x01020304 |
//   uint64 payload bytes | payload | uint64 FNV-1a (64-bit) of the payload
//
// with the payload a sequence of plain little-endian fields and arrays, in the order the writer
// put them.  The reader checks tag, version, byte order, size and checksum before anything is
// parsed, so a truncated or altered file is an error, never a partial object.
#pragma once
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.h"

namespace msasm {

constexpr uint32_t kStoreVersion = 1;
constexpr uint32_t kStoreByteOrder = 0x01020304u;

// FNV-1a, 64-bit: offset basis 14695981039346656037, prime 1099511628211
inline uint64_t fnv1a64(const unsigned char* p, size_t n) {
  uint64_t h = 14695981039346656037ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= uint64_t(p[i]);
    h *= 1099511628211ull;
  }
  return h;
}

class StoreWriter {
 public:
  template <typename T>
  void put(const T& v) {
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
    buf_.insert(buf_.end(), p, p + sizeof(T));
  }
  template <typename T>
  void put_array(const T* v, size_t n) {
    const unsigned char* p = reinterpret_cast<const unsigned char*>(v);
    buf_.insert(buf_.end(), p, p + n * sizeof(T));
  }
  // grow by n elements of T and return where they go (for device-to-host copies)
  template <typename T>
  T* reserve_array(size_t n) {
    const size_t at = buf_.size();
    buf_.resize(at + n * sizeof(T));
    return reinterpret_cast<T*>(buf_.data() + at);
  }
  size_t size() const { return buf_.size(); }
  unsigned char* at(size_t off) { return buf_.data() + off; }

  msasm_status write(const char* path, const char tag[8]) const {
    if (!path) return fail(MSASM_EINVAL, "path is NULL");
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(MSASM_EIO, std::string("cannot open for writing: ") + path);
    const uint64_t n = buf_.size(), h = fnv1a64(buf_.data(), buf_.size());
    bool ok = std::fwrite(tag, 1, 8, f) == 8;
    ok = ok && std::fwrite(&kStoreVersion, 4, 1, f) == 1 && std::fwrite(&kStoreByteOrder, 4, 1, f) == 1;
    ok = ok && std::fwrite(&n, 8, 1, f) == 1;
    ok = ok && (n == 0 || std::fwrite(buf_.data(), 1, n, f) == n);
    ok = ok && std::fwrite(&h, 8, 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(MSASM_EIO, std::string("write failed: ") + path);
    return MSASM_OK;
  }

 private:
  std::vector<unsigned char> buf_;
};

class StoreReader {
 public:
  // read and verify the whole file; get()/get_array() then walk the payload
  msasm_status open(const char* path, const char tag[8]) {
    if (!path) return fail(MSASM_EINVAL, "path is NULL");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(MSASM_EIO, std::string("cannot open: ") + path);
    char t[8];
    uint32_t version = 0, bom = 0;
    uint64_t n = 0, h = 0;
    bool ok = std::fread(t, 1, 8, f) == 8 && std::fread(&version, 4, 1, f) == 1 && std::fread(&bom, 4, 1, f) == 1 &&
              std::fread(&n, 8, 1, f) == 1;
    if (ok && std::memcmp(t, tag, 8) != 0) {
      std::fclose(f);
      return fail(MSASM_EIO, std::string("not a file of this kind (tag ") + std::string(tag, 8) + "): " + path);
    }
    if (ok && (version != kStoreVersion || bom != kStoreByteOrder)) {
      std::fclose(f);
      return fail(MSASM_EIO, std::string("unsupported format version or byte order: ") + path);
    }
    // the payload must fit the file: compare with the bytes left before allocating
    long here = ok ? std::ftell(f) : -1;
    ok = ok && here >= 0 && std::fseek(f, 0, SEEK_END) == 0;
    long end = ok ? std::ftell(f) : -1;
    ok = ok && end >= here && uint64_t(end - here) == n + 8 && std::fseek(f, here, SEEK_SET) == 0;
    if (ok) {
      try {
        buf_.resize(n);
      } catch (const std::bad_alloc&) {
        std::fclose(f);
        return fail(MSASM_ENOMEM, std::string("no host memory for the file: ") + path);
      }
      ok = (n == 0 || std::fread(buf_.data(), 1, n, f) == n) && std::fread(&h, 8, 1, f) == 1;
    }
    std::fclose(f);
    if (!ok) return fail(MSASM_EIO, std::string("truncated or unreadable file: ") + path);
    if (fnv1a64(buf_.data(), buf_.size()) != h) return fail(MSASM_EIO, std::string("checksum mismatch: ") + path);
    pos_ = 0;
    return MSASM_OK;
  }
  template <typename T>
  bool get(T& v) {
    if (buf_.size() - pos_ < sizeof(T)) return false;
    std::memcpy(&v, buf_.data() + pos_, sizeof(T));
    pos_ += sizeof(T);
    return true;
  }
  // pointer to n elements of T in the payload (unaligned: copy out with memcpy or cudaMemcpy)
  template <typename T>
  const unsigned char* get_array(size_t n) {
    if (n > (buf_.size() - pos_) / sizeof(T)) return nullptr;
    const unsigned char* p = buf_.data() + pos_;
    pos_ += n * sizeof(T);
    return p;
  }
  bool at_end() const { return pos_ == buf_.size(); }

 private:
  std::vector<unsigned char> buf_;
  size_t pos_ = 0;
};

}  // namespace msasm
