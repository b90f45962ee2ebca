// cg_snapshot.cpp -- save a context's checking state to a file and restore
// it into a fresh context: the allocation list with every allocation's
// device V shadow, the freed bases, the device arrays with their shadows
// and the destroyed array handles.  The host shadow image is the caller's
// and is not part of a snapshot.
//
// File layout (little-endian, 8-byte fields):
//   "CGSNAP01"
//   n_allocs,  then per allocation (ascending base): base, size, shadow bytes
//   n_freed,   then the freed bases
//   n_arrays,  then per array: handle, width, height, depth, shadow bytes
//   n_destroyed, then the destroyed array handles
#include <cuda_runtime.h>

#include <cstdio>

#include "cg_ctx.h"

using namespace cgi;

namespace {

constexpr char kMagic[8] = {'C', 'G', 'S', 'N', 'A', 'P', '0', '1'};
constexpr uint64_t kChunk = 32ull << 20;  // pinned staging per copy

struct File {
  std::FILE *f = nullptr;
  ~File() {
    if (f) std::fclose(f);
  }
};

struct Stage {
  PinBuf<uint8_t> buf;
  ~Stage() { buf.release(); }
};

cg_status io_fail(const char *what) {
  return set_error(CG_E_ARG, std::string("snapshot file: ") + what);
}

cg_status put(std::FILE *f, uint64_t v) {
  return std::fwrite(&v, 8, 1, f) == 1 ? CG_OK : io_fail("write failed");
}

cg_status get(std::FILE *f, uint64_t *v) {
  return std::fread(v, 8, 1, f) == 1 ? CG_OK : io_fail("truncated or unreadable");
}

// Device bytes [dev, dev+n) -> file, through pinned staging.
cg_status dump(std::FILE *f, PinBuf<uint8_t> &stage, uint64_t dev, uint64_t n) {
  for (uint64_t off = 0; off < n; off += kChunk) {
    const uint64_t k = std::min(kChunk, n - off);
    CG_CUDA(cudaMemcpy(stage.p, reinterpret_cast<const void *>(dev + off), k,
                       cudaMemcpyDeviceToHost));
    if (std::fwrite(stage.p, 1, k, f) != k) return io_fail("write failed");
  }
  return CG_OK;
}

// File -> device bytes [dev, dev+n).
cg_status load(std::FILE *f, PinBuf<uint8_t> &stage, uint64_t dev, uint64_t n) {
  for (uint64_t off = 0; off < n; off += kChunk) {
    const uint64_t k = std::min(kChunk, n - off);
    if (std::fread(stage.p, 1, k, f) != k) return io_fail("truncated or unreadable");
    CG_CUDA(cudaMemcpy(reinterpret_cast<void *>(dev + off), stage.p, k, cudaMemcpyHostToDevice));
  }
  return CG_OK;
}

}  // namespace

extern "C" {

cg_status cg_snapshot(cg_ctx *c, const char *path) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || !path) return set_error(CG_E_ARG, "NULL argument");
  CG_TRY(flush_fills(c, 0));
  CG_CUDA(cudaDeviceSynchronize());
  File F;
  F.f = std::fopen(path, "wb");
  if (!F.f) return io_fail("cannot open for writing");
  Stage S;
  CG_TRY(S.buf.ensure(kChunk));
  PinBuf<uint8_t> &stage = S.buf;
  if (std::fwrite(kMagic, 1, 8, F.f) != 8) return io_fail("write failed");
  c->table.merge();
  const AllocTable &t = c->table;
  CG_TRY(put(F.f, t.live));
  for (size_t j = 0; j < t.base.size(); j++) {
    if (!t.size[j]) continue;
    CG_TRY(put(F.f, t.base[j]));
    CG_TRY(put(F.f, t.size[j]));
    CG_TRY(dump(F.f, stage, t.shadow[j], t.size[j]));
  }
  CG_TRY(put(F.f, t.freed.size()));
  for (uint64_t b : t.freed) CG_TRY(put(F.f, b));
  CG_TRY(put(F.f, c->arrays.size()));
  for (const auto &kv : c->arrays) {
    const cg_ctx::ArrayInfo &a = kv.second;
    CG_TRY(put(F.f, kv.first));
    CG_TRY(put(F.f, a.w));
    CG_TRY(put(F.f, a.h));
    CG_TRY(put(F.f, a.d));
    CG_TRY(dump(F.f, stage, a.shadow, a.w * a.h * a.d));
  }
  CG_TRY(put(F.f, c->freed_arrays.size()));
  for (uint64_t h : c->freed_arrays) CG_TRY(put(F.f, h));
  if (std::fflush(F.f) != 0) return io_fail("write failed");
  return CG_OK;
}

cg_status cg_restore(cg_ctx *c, const char *path) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || !path) return set_error(CG_E_ARG, "NULL argument");
  if (c->table.live || !c->table.freed.empty() || !c->arrays.empty() || !c->freed_arrays.empty())
    return set_error(CG_E_STATE, "restore needs a context with no allocations or arrays");
  File F;
  F.f = std::fopen(path, "rb");
  if (!F.f) return io_fail("cannot open for reading");
  char magic[8];
  if (std::fread(magic, 1, 8, F.f) != 8 || std::memcmp(magic, kMagic, 8) != 0)
    return io_fail("not a libcg snapshot");
  Stage S;
  CG_TRY(S.buf.ensure(kChunk));
  PinBuf<uint8_t> &stage = S.buf;
  CG_TRY(flush_fills(c, 0));
  uint64_t n = 0;
  CG_TRY(get(F.f, &n));
  for (uint64_t i = 0; i < n; i++) {
    uint64_t b, s;
    CG_TRY(get(F.f, &b));
    CG_TRY(get(F.f, &s));
    CG_TRY(cg_register_alloc(c, b, s));
    CG_TRY(load(F.f, stage, c->table.find(b).shadow, s));
  }
  CG_TRY(get(F.f, &n));
  for (uint64_t i = 0; i < n; i++) {
    uint64_t b;
    CG_TRY(get(F.f, &b));
    c->table.freed.insert(b);
  }
  CG_TRY(get(F.f, &n));
  for (uint64_t i = 0; i < n; i++) {
    uint64_t h, w, ht, d;
    CG_TRY(get(F.f, &h));
    CG_TRY(get(F.f, &w));
    CG_TRY(get(F.f, &ht));
    CG_TRY(get(F.f, &d));
    CG_TRY(cg_register_array(c, h, w, ht, d));
    CG_TRY(load(F.f, stage, c->arrays[h].shadow, w * ht * d));
  }
  CG_TRY(get(F.f, &n));
  for (uint64_t i = 0; i < n; i++) {
    uint64_t h;
    CG_TRY(get(F.f, &h));
    c->freed_arrays.insert(h);
  }
  c->table.dev_stale();  // the device copy of the table is rebuilt on next use
  return CG_OK;
}

}  // extern "C"
