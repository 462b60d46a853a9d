/*
 * qp_gb300.h -- C ABI of the batched differentiable QP solver (OptNet hot path) for
 * NVIDIA GB300 (sm_103a).
 *
 * Problem (Amos & Kolter 2017, §3, Eq. 2), one per batch instance:
 *
 *     minimise_z  ½ zᵀ Q z + qᵀ z   subject to   A z = b,  G z ≤ h
 *
 * with z ∈ Rⁿ, G ∈ R^{nineq×n}, A ∈ R^{neq×n}.  The paper writes A with m rows and G with
 * p rows; this ABI names the row counts `nineq` (rows of G) and `neq` (rows of A).
 *
 * Layout: every matrix and vector argument is a DEVICE pointer to dense, row-major,
 * batch-major data (instance b of Q starts at Q + b·n·n, of G at G + b·nineq·n, ...),
 * of the element type chosen by `dtype`.  Q must be symmetric positive semidefinite, and the
 * KKT system nonsingular at the solution (Q positive definite on the null space of the
 * active constraints and of A, A of full row rank).
 * Pointers must be aligned to the element size.  All calls are asynchronous on `stream`
 * (a cudaStream_t, NULL = legacy default stream) and never synchronise the host.
 *
 * Ownership: the library never allocates device memory in these calls.  The caller owns
 * every buffer, including the workspace that carries the factorisation from
 * qp_forward to qp_backward (size from qp_workspace_bytes).
 *
 * Errors: call-level problems return a QP_E* code and launch nothing.  Per-instance
 * numerical outcomes are reported in status[b] (QP_STATUS_*); kernels never trap.
 */
#ifndef QP_GB300_H
#define QP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define QP_OK            0
#define QP_EINVAL        1  /* null pointer, negative size, bad dtype, B = 0 allowed */
#define QP_ENOSPACE      2  /* workspace smaller than qp_workspace_bytes()          */
#define QP_EUNSUPPORTED  3  /* sizes beyond what the kernels of this build handle   */
#define QP_ECUDA         4  /* a CUDA launch or attribute call failed               */

/* Element types. */
#define QP_F32 0  /* FP32 matrices and factors; FP64-accurate residuals and iterate */
#define QP_F64 1  /* everything in FP64                                              */

/* Per-instance status codes written to status[b] by the forward pass, and status words
 * written by the backward pass when it is given a status array: the low 8 bits hold the code,
 * higher bits are flags (QP_STATUS_CODE(s) extracts the code; forward statuses carry no
 * flags). */
#define QP_STATUS_CONVERGED 0  /* residual and duality tests met                          */
#define QP_STATUS_MAX_ITER  1  /* max_iter Newton steps taken; iterate returned anyway   */
#define QP_STATUS_NOT_PD    2  /* a pivot of Q, of A Q⁻¹Aᵀ or of the per-iteration Schur
                                  complement was not positive: outputs are NaN          */
#define QP_STATUS_NUMERICAL 3  /* a non-finite value appeared: outputs are NaN           */
#define QP_STATUS_NO_FORWARD 4 /* backward only: the workspace holds no forward pass of this
                                  instance (no stamp, other sizes, dtype, kernel path or
                                  Q/G/A buffers): gradients are NaN                     */
#define QP_STATUS_INFEASIBLE 5 /* infeasibility suspected: the returned λ ≥ 0, ν satisfy
                                  −(hᵀλ + bᵀν) > 1e3·(1 + ‖z‖∞)·‖Gᵀλ + Aᵀν‖₁, so by Farkas'
                                  lemma any feasible point has ‖z'‖∞ > 1e3·(1 + ‖z‖∞).
                                  z, λ, ν are returned, λ and ν scaled so that
                                  max(‖λ‖∞, ‖ν‖∞) = 1: they are the certificate.  Checked
                                  once ‖λ‖∞ passes 1e3 × its first-iteration value, and
                                  when the loop ends on max_iter, the time limit or a
                                  Newton system that is no longer positive definite.
                                  Gradients are NaN                                      */
#define QP_STATUS_TIMEOUT   6  /* the time limit of qp_options ran out; iterate returned
                                  as for MAX_ITER                                        */
#define QP_STATUS_CODE(s) ((s) & 0xff)
/* Flag bit of backward status words: at the returned iterate some complementarity pair has
 * max(λ_i, s_i) ≤ 1e-5·max(1, max_j max(λ_j, s_j)), a nearly degenerate point where the
 * proof of Theorem 1 no longer gives a unique derivative (the gradient returned there is
 * one element of a set). */
#define QP_FLAG_NEAR_DEGENERATE 0x100
/* Flag bit of backward status words: Q was only positive semidefinite (a pivot of Q in the
 * setup fell below 1e-5, FP64 1e-12, of max_i Q_ii), so the factorisations used Q + δI with
 * δ = 1e-4 (FP64 1e-8) × max(max_i Q_ii, squared row norms of G and A); the KKT residual that
 * drives the iteration and the backward refinement use Q itself, so the results are those of
 * the QP with Q. */
#define QP_FLAG_REGULARIZED_Q 0x200

typedef struct qp_options {
  double  tol;       /* stop when ‖r_z‖∞ ≤ tol·(1+‖q‖∞), ‖Gz+s−h‖∞ ≤ tol·(1+‖h‖∞),
                        ‖Az−b‖∞ ≤ tol·(1+‖b‖∞) ...                                   */
  double  mu_tol;    /* ... and μ = sᵀλ/nineq ≤ mu_tol                                */
  int32_t max_iter;  /* bound on Newton steps of the interior point loop               */
  int32_t refine;    /* most FP64 iterative-refinement steps of the backward KKT solve
                        (0-4); refinement stops once each block of the correction is
                        below 1e-3 of its block of the solution (floored at 1e-6 of
                        ‖∂ℓ/∂z*‖∞): one step for well-conditioned systems            */
  int32_t path;      /* 0: automatic kernel choice; 1: always the global-memory kernel.
                        Forward and backward of one batch must use the same value.      */
  int32_t time_limit_us; /* forward only: an instance still iterating this many
                        microseconds after its block started stops with status
                        QP_STATUS_TIMEOUT (0 = no limit)                                */
} qp_options;

/* Default options for a dtype (QP_F32: tol 1e-10, mu_tol 1e-11, max_iter 50, refine 4;
 * QP_F64: tol 1e-12, mu_tol 1e-13, max_iter 100, refine 4; path 0, no time limit). */
void qp_default_options(int dtype, qp_options* opt);

/* Bytes of workspace qp_forward needs for B instances of one size (0 on invalid sizes),
 * for the automatic kernel choice (qp_workspace_bytes_opt: for the given options). */
size_t qp_workspace_bytes(int dtype, int B, int n, int nineq, int neq);
size_t qp_workspace_bytes_opt(const qp_options* opt, int dtype, int B, int n, int nineq,
                              int neq);

/* QP_OK if this build's kernels handle the size, else QP_EUNSUPPORTED / QP_EINVAL. */
int qp_supported(int dtype, int n, int nineq, int neq);

/* 1 if instances of this size run on the global-memory kernel (factors kept in the
 * workspace, L2-resident), 0 if on the shared-memory kernel, −1 on invalid arguments. */
int qp_uses_global_path(int dtype, int n, int nineq, int neq);

/* 1 if qp_forward's setup factorisation of this size (§3.1: the blocks of the KKT matrix that
 * do not change over the iterations, factored once) runs its rank-64 updates on the tensor
 * cores (tcgen05, TF32 with a three-term split that keeps FP32 accuracy): FP32 instances on
 * the global-memory kernel with n + neq ≥ 128 (after padding) whose operand tiles fit in
 * shared memory.  0 otherwise (the CUDA-core sweep), −1 on invalid arguments.  `opt` may be
 * NULL (automatic path) or force the path as qp_forward would.  The packed entry points
 * always use the CUDA-core sweep. */
int qp_uses_tensor_cores(const qp_options* opt, int dtype, int n, int nineq, int neq);

/*
 * qp_forward -- batched primal-dual interior point solve (§3.1: slack form, affine
 * predictor Eq. 9, centering-plus-corrector Eq. 10, symmetrised and block-eliminated KKT
 * system with the parts that do not involve D(λ/s) factored once).
 *
 * In:   Q [B,n,n], q [B,n], G [B,nineq,n], h [B,nineq], A [B,neq,n], b [B,neq].
 *       G/h may be NULL when nineq = 0, A/b may be NULL when neq = 0.
 * Out:  z [B,n] = z*, lam [B,nineq] = λ*, nu [B,neq] = ν* (lam/nu may be NULL when their
 *       size is 0), status [B] (QP_STATUS_*), iters [B] (Newton steps taken), and
 *       optionally resid [B,4] (FP64): ‖Qz+q+Gᵀλ+Aᵀν‖∞, ‖Gz+s−h‖∞, ‖Az−b‖∞ and
 *       μ = sᵀλ/nineq at the returned iterate (status/iters/resid may be NULL).
 * Work: workspace of at least qp_workspace_bytes(dtype,B,n,nineq,neq) bytes, 256-byte
 *       aligned; it keeps the factorisation at the returned iterate and the FP64 iterate
 *       for qp_backward.  It must not be modified between the two calls.  Each instance's
 *       slot ends with a stamp (a magic word, the sizes, dtype, kernel path and a hash of
 *       the instance's Q/G/A addresses) that qp_backward checks on the device.
 * opt:  NULL = qp_default_options(dtype).
 */
int qp_forward(const qp_options* opt, int dtype, int B, int n, int nineq, int neq,
               const void* Q, const void* q, const void* G, const void* h,
               const void* A, const void* b,
               void* z, void* lam, void* nu, int32_t* status, int32_t* iters,
               double* resid, void* workspace, size_t workspace_bytes, void* stream);

/*
 * qp_backward -- gradients of ℓ(z*) through the KKT conditions (§3, Eq. 7 and Eq. 8),
 * computed as in §3.1.1 (Eq. 11) with the factorisation qp_forward left in `workspace`:
 * K_sym [d_z; d_s; d̃_λ; d_ν] = [−∂ℓ/∂z*; 0; 0; 0], then
 *   dQ = ½(d_z z*ᵀ + z* d_zᵀ), dq = d_z, dG = d̃_λ z*ᵀ + λ* d_zᵀ, dh = −d̃_λ,
 *   dA = d_ν z*ᵀ + ν* d_zᵀ,    db = −d_ν.
 * Up to `refine` steps of iterative refinement with an FP64-accurate KKT residual follow
 * the first solve (see qp_options).  Q, G, A must be the same buffers, holding the same
 * data, as passed to qp_forward (they feed the refinement residual).  dl_dz [B,n] is
 * ∂ℓ/∂z*.  Any gradient pointer may be NULL (not wanted).  Instances whose forward status
 * was NOT_PD, NUMERICAL or INFEASIBLE get NaN gradients; so do instances whose workspace
 * stamp does not match this call (no forward of these sizes, dtype, kernel path and Q/G/A
 * buffers ran on it: QP_STATUS_NO_FORWARD).  A stamp cannot tell whether the data in the
 * buffers changed since the forward pass.  Call-level errors as qp_forward (the host
 * checks the workspace size); nothing is synchronised.
 */
int qp_backward(const qp_options* opt, int dtype, int B, int n, int nineq, int neq,
                const void* Q, const void* G, const void* A,
                const void* workspace, size_t workspace_bytes, const void* dl_dz,
                void* dQ, void* dq, void* dG, void* dh, void* dA, void* db, void* stream);

/*
 * qp_backward_ext -- qp_backward for a loss that also depends on λ* and ν*, with an
 * optional per-instance status output.
 *
 * §3 differentiates z* only (it sets the λ*, ν* case aside).  The same implicit
 * differentiation of Eq. 6 gives, for a loss of (z*, λ*, ν*), the adjoint of Eq. 7 with
 * right-hand side [∂ℓ/∂z*; ∂ℓ/∂λ*; ∂ℓ/∂ν*] instead of [∂ℓ/∂z*; 0; 0], and the gradients of
 * Eq. 8 unchanged.  In the symmetrised form of Eq. 11 the two new blocks enter the primal
 * feasibility rows: K_sym [d_z; d_s; d̃_λ; d_ν] = [−∂ℓ/∂z*; 0; −∂ℓ/∂λ*; −∂ℓ/∂ν*].
 *
 * dl_dlam: [B, nineq] and dl_dnu: [B, neq], device memory of the dtype, row-major; either
 * may be null (zero).  dl_dz is required (pass zeros for a loss of λ*, ν* alone).
 * status: [B] int32 device memory or NULL; receives the forward pass's status code of each
 * instance, or QP_STATUS_NO_FORWARD when its workspace stamp does not match.  All other
 * arguments, outputs and errors as qp_backward; qp_backward(...) is this call with
 * dl_dlam, dl_dnu and status null.
 */
int qp_backward_ext(const qp_options* opt, int dtype, int B, int n, int nineq, int neq,
                    const void* Q, const void* G, const void* A,
                    const void* workspace, size_t workspace_bytes, const void* dl_dz,
                    const void* dl_dlam, const void* dl_dnu,
                    void* dQ, void* dq, void* dG, void* dh, void* dA, void* db,
                    int32_t* status, void* stream);

/*
 * Packed batches of uneven sizes (one persistent launch each way).
 *
 * Instance i has its own (n_i, nineq_i, neq_i); its data are packed back to back in index
 * order in each input buffer (Q_i n_i×n_i row-major, then Q_{i+1}, ...; likewise q, G, h, A,
 * b, the outputs z, λ, ν and the gradients, which share the inputs' offsets).  The
 * paper's solver is stated for fixed-size batches (§3.1); this entry runs the same method
 * per instance, each on the kernel path its own size selects, so an instance's result does
 * not depend on the rest of the batch.
 */
typedef struct qp_instance_desc {
  int32_t n, nineq, neq;     /* sizes                                                   */
  int32_t id;                /* index of the instance (status/iters/resid slots)        */
  int32_t nz;                /* n plus dummy padding (set by qp_packed_plan)            */
  int32_t flags;             /* bit 0: global-memory kernel (set by qp_packed_plan)     */
  int64_t oQ, oq, oG, oh, oA, ob;   /* element offsets into the packed inputs/gradients */
  int64_t oz, olam, onu;            /* element offsets into the packed outputs          */
  int64_t ows;                      /* byte offset of the instance's workspace          */
} qp_instance_desc;

typedef struct qp_packed_sizes {
  int64_t nQ, nq, nG, nh, nA, nb;   /* elements of each packed input (= its gradient)   */
  int64_t nz, nlam, nnu;            /* elements of each packed output                   */
  int64_t ws_bytes;                 /* workspace bytes, 256-byte aligned                */
  int64_t fwd_smem, bwd_smem;       /* dynamic shared memory of the packed kernels      */
  int32_t sw, ch;                   /* register-tile variant of the shared-memory path  */
  int32_t n_global;                 /* instances on the global-memory path              */
  int32_t reserved;
} qp_packed_sizes;

/* Host-side planning: dims is a HOST array of B triples (n, nineq, neq).  Fills the HOST
 * arrays desc[B] (in execution order: the sizes->n_global global-path instances first, then
 * the shared-memory-path ones, each part largest estimated cost first) and *sizes.  The
 * caller copies desc to device memory unchanged and passes it, with sizes, to the packed
 * calls. */
int qp_packed_plan(const qp_options* opt, int dtype, int B, const int32_t* dims,
                   qp_instance_desc* desc, qp_packed_sizes* sizes);

/* qp_packed_plan with per-instance hints from a tuner: path_hint[i] (may be NULL) is 0 for
 * the automatic choice, 1 for the global-memory kernel, 2 for the shared-memory kernel
 * (QP_EUNSUPPORTED if it cannot take that size); cost[i] (may be NULL) replaces the built-in
 * cost estimate that orders the work queue (largest first). */
int qp_packed_plan_ex(const qp_options* opt, int dtype, int B, const int32_t* dims,
                      const int8_t* path_hint, const float* cost, qp_instance_desc* desc,
                      qp_packed_sizes* sizes);

/* Forward pass of a packed batch (device pointers as in qp_forward, packed as above;
 * status/iters/resid indexed by instance id; workspace of sizes->ws_bytes bytes).  When a
 * batch holds both kinds, the global-path and shared-memory-path instances run as two
 * persistent kernels side by side: the global-path one first, on `stream`, the other on a
 * library-owned side stream forked from `stream` and joined back to it by events (one side
 * stream per caller stream, for up to 16 streams per device; created on a stream's first
 * such call: make that call before any stream capture).  Its blocks take SMs as the
 * global-path blocks finish their queue. */
int qp_forward_packed(const qp_options* opt, int dtype, int B, const qp_instance_desc* desc,
                      const qp_packed_sizes* sizes, const void* Q, const void* q,
                      const void* G, const void* h, const void* A, const void* b, void* z,
                      void* lam, void* nu, int32_t* status, int32_t* iters, double* resid,
                      void* workspace, size_t workspace_bytes, void* stream);

/* Backward pass of a packed batch, after qp_forward_packed with the same desc, sizes and
 * workspace.  dl_dz is packed like z; the gradients like the inputs.  It differentiates a
 * loss of z* (for a loss that also depends on λ*, ν*, use qp_backward_ext on a fixed-size
 * batch).  status (int32 [B] indexed by instance id, or NULL) as in qp_backward_ext.  The
 * workspace is written: bytes 4..7 hold the backward pass's work-queue counter, so two
 * backward calls on one workspace must not overlap on the GPU. */
int qp_backward_packed(const qp_options* opt, int dtype, int B, const qp_instance_desc* desc,
                       const qp_packed_sizes* sizes, const void* Q, const void* G,
                       const void* A, void* workspace, size_t workspace_bytes,
                       const void* dl_dz, void* dQ, void* dq, void* dG, void* dh, void* dA,
                       void* db, int32_t* status, void* stream);

/*
 * qp_forward_noalloc -- qp_forward for callers that cannot allocate device memory (a control
 * loop with a hard latency budget, a process whose device memory is fixed when it starts, a
 * plugin whose host framework owns all allocation).  The paper has no counterpart: this is an
 * interface variant, not part of the method.
 *
 * Same arguments and results as qp_forward, but no workspace: the library's own file-scope
 * device array of QP_NOALLOC_SCRATCH_BYTES bytes (32 MiB, held by every device that loads the
 * library until exit) takes its place.  It allocates nothing.  Returns QP_ENOSPACE when
 * qp_workspace_bytes_opt() for the call exceeds QP_NOALLOC_SCRATCH_BYTES (e.g. about 170
 * instances of n = 100, nineq = 100, neq = 50 in FP32).  The first call on a device looks up
 * the array's address there (make it before any stream capture) and caches it for the life of
 * the process; after a cudaDeviceReset of that device the cached address is stale, so do not
 * call this entry point on a device that was reset.  All calls share the
 * array, so calls that overlap on the GPU race; its contents after a call are that call's
 * factorisation, which is not reachable from qp_backward.
 */
#define QP_NOALLOC_SCRATCH_BYTES (32u << 20)
int qp_forward_noalloc(const qp_options* opt, int dtype, int B, int n, int nineq, int neq,
                       const void* Q, const void* q, const void* G, const void* h,
                       const void* A, const void* b, void* z, void* lam, void* nu,
                       int32_t* status, int32_t* iters, double* resid, void* stream);

/* Human-readable text for a QP_E* code. */
const char* qp_strerror(int code);

/* qp_host_copy_many -- host-side utility of the serving loop; the paper has no counterpart.
 * Copies `count` host buffers: bytes[i] bytes from src[i] to dst[i], for i < count, on up to
 * `threads` host threads (one thread for small totals).  All pointers are host memory owned
 * by the caller; source and destination ranges must not overlap.  It touches no GPU state.
 * Returns QP_OK, or QP_EINVAL for a negative count or null arrays. */
int qp_host_copy_many(int count, void* const* dst, const void* const* src,
                      const size_t* bytes, int threads);

/* Field rules of qp_host_pack / qp_host_unpack: the length and packed offset of one
 * instance's array, from its descriptor (outputs share the rules of the inputs they are
 * laid out like: z and ∂ℓ/∂z* like q, λ like h, ν like b, gradients like their inputs). */
#define QP_FIELD_Q 0   /* n·n at oQ      */
#define QP_FIELD_Q1 1  /* n at oq        */
#define QP_FIELD_G 2   /* nineq·n at oG  */
#define QP_FIELD_H 3   /* nineq at oh    */
#define QP_FIELD_A 4   /* neq·n at oA    */
#define QP_FIELD_B 5   /* neq at ob      */

/* qp_host_pack -- host-side utility of the serving loop; the paper has no counterpart.
 * Gathers per-instance HOST arrays into one packed HOST buffer laid out as the packed calls
 * expect.  desc[B]: a plan from qp_packed_plan (any order; ids 0..B−1).  For each instance
 * and each field f < nfields, copies src[id·nfields + f] (len elements of esz bytes, by rule
 * fields[f]; a NULL source is skipped) to dst + (sec[f] + off)·esz, off the rule's packed
 * offset.  sec[f] is the element offset of field f's section in dst.  Runs on up to
 * `threads` host threads; touches no GPU state.  QP_EINVAL on bad arguments. */
int qp_host_pack(int B, const qp_instance_desc* desc, int esz, int nfields,
                 const int32_t* fields, const int64_t* sec, const void* const* src, void* dst,
                 int threads);

/* qp_host_unpack -- the inverse gather for results: reads field f of each instance from
 * src + (sec[f] + off)·esz and writes instance id's fields contiguously, in field order, to
 * dst + dst_off[id]·esz; fills dst_off[0..B] (dst_off[B] = total elements).  dst must hold
 * dst_off[B] elements (at most B·Σ field lengths of the largest instance; callers size it
 * from the plan totals: Σ_f sizes of the sections).  Host memory only. */
int qp_host_unpack(int B, const qp_instance_desc* desc, int esz, int nfields,
                   const int32_t* fields, const int64_t* sec, const void* src, void* dst,
                   int64_t* dst_off, int threads);

#ifdef __cplusplus
}
#endif
#endif /* QP_GB300_H */
