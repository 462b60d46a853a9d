// Runs qp_forward + qp_backward_ext of the C ABI, compiled for the host with the emulation
// shims, on one input file, and writes the results.
// Input: int32 B, n, nineq, neq, dtype, path; then Q, q, G, h, A, b, dl_dz of the dtype.
// Output: z, lam, nu, dQ, dq, dG, dh, dA, db, then int32 status[B], backward status[B].
#include <cstdio>
#include <cstdlib>
#include <cstring>

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
  if (argc < 3) {
    fprintf(stderr, "usage: driver in.bin out.bin\n");
    return 2;
  }
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t hdr[6];
  if (fread(hdr, 4, 6, f) != 6) return 2;
  const int B = hdr[0], n = hdr[1], p = hdr[2], m = hdr[3], dtype = hdr[4];
  const size_t es = dtype == QP_F32 ? 4 : 8;
  const size_t cnt[7] = {(size_t)B * n * n, (size_t)B * n, (size_t)B * p * n, (size_t)B * p,
                         (size_t)B * m * n, (size_t)B * m, (size_t)B * n};
  void* in[7];
  for (int k = 0; k < 7; ++k) {
    in[k] = xalloc(cnt[k] * es, 0);
    if (cnt[k] && fread(in[k], es, cnt[k], f) != cnt[k]) return 2;
  }
  fclose(f);
  qp_options o;
  qp_default_options(dtype, &o);
  o.path = hdr[5];
  const size_t wsb = qp_workspace_bytes_opt(&o, dtype, B, n, p, m);
  void* ws = xalloc(wsb, 0xff);   // as uninitialised as device memory may be
  void* z = xalloc((size_t)B * n * es, 0);
  void* lam = xalloc((size_t)B * p * es, 0);
  void* nu = xalloc((size_t)B * m * es, 0);
  int32_t* st = (int32_t*)xalloc(4 * B, 0xff);
  int32_t* it = (int32_t*)xalloc(4 * B, 0xff);
  double* resid = (double*)xalloc(32 * B, 0xff);
  int rc = qp_forward(&o, dtype, B, n, p, m, in[0], in[1], p ? in[2] : nullptr,
                      p ? in[3] : nullptr, m ? in[4] : nullptr, m ? in[5] : nullptr, z,
                      p ? lam : nullptr, m ? nu : nullptr, st, it, resid, ws, wsb, nullptr);
  if (rc != QP_OK) {
    fprintf(stderr, "qp_forward: %d\n", rc);
    return 3;
  }
  void* g[6];
  for (int k = 0; k < 6; ++k) g[k] = xalloc(cnt[k] * es, 0xff);
  int32_t* bst = (int32_t*)xalloc(4 * B, 0xff);
  rc = qp_backward_ext(&o, dtype, B, n, p, m, in[0], p ? in[2] : nullptr, m ? in[4] : nullptr, ws,
                       wsb, in[6], nullptr, nullptr, g[0], g[1], p ? g[2] : nullptr,
                       p ? g[3] : nullptr, m ? g[4] : nullptr, m ? g[5] : nullptr, bst, nullptr);
  if (rc != QP_OK) {
    fprintf(stderr, "qp_backward_ext: %d\n", rc);
    return 3;
  }
  FILE* out = fopen(argv[2], "wb");
  fwrite(z, es, (size_t)B * n, out);
  fwrite(lam, es, (size_t)B * p, out);
  fwrite(nu, es, (size_t)B * m, out);
  for (int k = 0; k < 6; ++k) fwrite(g[k], es, cnt[k], out);
  fwrite(st, 4, B, out);
  fwrite(bst, 4, B, out);
  fclose(out);
  return 0;
}
