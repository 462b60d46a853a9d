// Runs qp_packed_plan + qp_forward_packed + qp_backward_packed of the C ABI, compiled for the
// host with the emulation shims, on one input file of mixed sizes, and writes the results.
// Input: int32 B, dtype; int32 dims[B][3] (n, nineq, neq); then per instance Q, q, G, h, A,
// b, dl_dz of the dtype.  Output, per instance in input order: z, lam, nu, dQ, dq, dG, dh,
// dA, db; then int32 status[B] and backward status[B].
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "qp_gb300.h"
#include "shim.h"

thread_local EmuDim3 threadIdx, blockIdx;
unsigned char* emu_dyn_smem = nullptr;
EmuBlock* emu_blk = nullptr;

static void* xalloc(size_t bytes, int fill) {
  void* p = nullptr;
  if (posix_memalign(&p, 256, bytes ? bytes : 1) != 0) abort();
  std::memset(p, fill, bytes ? bytes : 1);
  return p;
}

int main(int argc, char** argv) {
  if (argc < 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t hdr[2];
  if (fread(hdr, 4, 2, f) != 2) return 2;
  const int B = hdr[0], dtype = hdr[1];
  const size_t es = dtype == QP_F32 ? 4 : 8;
  std::vector<int32_t> dims(3 * (size_t)B);
  if (fread(dims.data(), 4, dims.size(), f) != dims.size()) return 2;
  qp_options o;
  qp_default_options(dtype, &o);
  std::vector<qp_instance_desc> desc(B);
  qp_packed_sizes S;
  int rc = qp_packed_plan(&o, dtype, B, dims.data(), desc.data(), &S);
  if (rc != QP_OK) { fprintf(stderr, "plan: %d\n", rc); return 3; }
  std::vector<int> slot(B);   // descriptor index of each instance id
  for (int k = 0; k < B; ++k) slot[desc[k].id] = k;
  const int64_t tot[6] = {S.nQ, S.nq, S.nG, S.nh, S.nA, S.nb};
  unsigned char* in[7];
  for (int k = 0; k < 6; ++k) in[k] = (unsigned char*)xalloc((size_t)tot[k] * es, 0);
  in[6] = (unsigned char*)xalloc((size_t)S.nq * es, 0);   // dl_dz, packed like q
  for (int i = 0; i < B; ++i) {
    const int n = dims[3 * i], p = dims[3 * i + 1], m = dims[3 * i + 2];
    const qp_instance_desc& d = desc[slot[i]];
    const size_t cnt[7] = {(size_t)n * n, (size_t)n, (size_t)p * n, (size_t)p, (size_t)m * n,
                           (size_t)m, (size_t)n};
    const int64_t off[7] = {d.oQ, d.oq, d.oG, d.oh, d.oA, d.ob, d.oq};
    for (int k = 0; k < 7; ++k)
      if (cnt[k] && fread(in[k] + (size_t)off[k] * es, es, cnt[k], f) != cnt[k]) return 2;
  }
  fclose(f);
  void* ws = xalloc((size_t)S.ws_bytes, 0xff);   // as uninitialised as device memory may be
  void* z = xalloc((size_t)S.nz * es, 0);
  void* lam = xalloc((size_t)S.nlam * es, 0);
  void* nu = xalloc((size_t)S.nnu * es, 0);
  int32_t* st = (int32_t*)xalloc(4 * (size_t)B, 0xff);
  int32_t* it = (int32_t*)xalloc(4 * (size_t)B, 0xff);
  double* resid = (double*)xalloc(32 * (size_t)B, 0xff);
  rc = qp_forward_packed(&o, dtype, B, desc.data(), &S, in[0], in[1], S.nG ? in[2] : nullptr,
                         S.nh ? in[3] : nullptr, S.nA ? in[4] : nullptr, S.nb ? in[5] : nullptr,
                         z, S.nlam ? lam : nullptr, S.nnu ? nu : nullptr, st, it, resid, ws,
                         (size_t)S.ws_bytes, nullptr);
  if (rc != QP_OK) { fprintf(stderr, "qp_forward_packed: %d\n", rc); return 3; }
  void* g[6];
  for (int k = 0; k < 6; ++k) g[k] = xalloc((size_t)tot[k] * es, 0);
  int32_t* bst = (int32_t*)xalloc(4 * (size_t)B, 0xff);
  rc = qp_backward_packed(&o, dtype, B, desc.data(), &S, in[0], S.nG ? in[2] : nullptr,
                          S.nA ? in[4] : nullptr, ws, (size_t)S.ws_bytes, in[6], g[0], g[1],
                          S.nG ? g[2] : nullptr, S.nh ? g[3] : nullptr, S.nA ? g[4] : nullptr,
                          S.nb ? g[5] : nullptr, bst, nullptr);
  if (rc != QP_OK) { fprintf(stderr, "qp_backward_packed: %d\n", rc); return 3; }
  FILE* out = fopen(argv[2], "wb");
  for (int i = 0; i < B; ++i) {
    const int n = dims[3 * i], p = dims[3 * i + 1], m = dims[3 * i + 2];
    const qp_instance_desc& d = desc[slot[i]];
    fwrite((unsigned char*)z + (size_t)d.oz * es, es, n, out);
    fwrite((unsigned char*)lam + (size_t)d.olam * es, es, p, out);
    fwrite((unsigned char*)nu + (size_t)d.onu * es, es, m, out);
    const size_t cnt[6] = {(size_t)n * n, (size_t)n, (size_t)p * n, (size_t)p, (size_t)m * n,
                           (size_t)m};
    const int64_t off[6] = {d.oQ, d.oq, d.oG, d.oh, d.oA, d.ob};
    for (int k = 0; k < 6; ++k) fwrite((unsigned char*)g[k] + (size_t)off[k] * es, es, cnt[k], out);
  }
  fwrite(st, 4, B, out);
  fwrite(bst, 4, B, out);
  fclose(out);
  return 0;
}
