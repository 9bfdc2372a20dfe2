// Kernel launchers of the sm_103a condensed spectral-element library.
#pragma once

#include <cuda_bf16.h>

#include "sem_internal.h"

// Storage type of the CG's inverse-diagonal (BT) preconditioner: T in the
// FP64 CG; BF16 in the FP32 inner CG of mixed-precision solves.  The
// preconditioner is a fixed diagonal scaling, so rounding each entry to BF16
// (relative change <= 2^-9) moves the spectrum of the preconditioned operator
// by a factor within 1 +- 2^-8 and keeps it SPD, and every CG step reads
// half the bytes for it.
template <typename T>
struct PrecStore {
  using type = T;
};
template <>
struct PrecStore<float> {
  using type = __nv_bfloat16;
};
template <typename T>
using prec_t = typename PrecStore<T>::type;

// Operator kernel variants: one operator, five work mappings (sem_apply.cu,
// sem_apply_plane.cu, sem_apply_slab.cu).  The numbering is the one of SEM_KERNEL_* in sem.h.
enum ApplyKind {
  kApplyAuto = 0,      // the built-in choice for (n, precision)
  kApplyCta = 1,       // CTA tile of epb elements, k-slabs of depth ks
  kApplyWarp = 2,      // one warp per element (FP32, 3 <= n <= 7)
  kApplyPlane = 3,     // lanes per y-plane: 32/G elements per warp (FP32, 2 <= n <= 8) or
                       // one element per warp, half rows (FP32, 9 <= n <= 15)
  kApplyElement = 4,   // one thread per element (n = 1; FP32 also n = 2, 3)
  kApplySlab = 5,      // element x slab of 8 planes k per CTA (FP32, 16 <= n <= 31)
  kApplyRow = 6,       // x-row segment of up to 32 elements per CTA, bulk copies (FP32, 2 <= n <= 8)
  kApplyPencil = 7     // thread per x-pencil, then per cube column (FP32, 5 <= n <= 8)
};

// Operator launch configuration.
struct ApplyConfig {
  int kind = kApplyAuto;
  int epb = 0;      // CTA tile: elements per tile
  int ks = 0;       // CTA tile: eigenspace slab depth (k planes held at once)
  int threads = 0;
  size_t smem = 0;  // CTA tile: dynamic shared memory bytes
  // Fixed-order edge and vertex sums (bitwise reproducible output): scratch of
  // nelem (12 n + 8) values of the operator's type, or null for atomics.
  void* ev = nullptr;
};
// Built-in CTA-tile shape for n.
ApplyConfig sem_apply_config(int n, size_t elem_bytes);
// Explicit CTA-tile configuration (autotuner candidates).
ApplyConfig sem_apply_config_make(int n, size_t elem_bytes, int epb, int ks);
// A configuration of the given kind (no tile parameters).
ApplyConfig sem_apply_config_kind(int kind);
// Whether c names a variant that exists for (n, element bytes) and, for a
// CTA tile, one that fits in shared memory.
bool sem_apply_config_valid(int n, size_t elem_bytes, const ApplyConfig& c);
// The kind kApplyAuto resolves to.
int sem_apply_default_kind(int n, size_t elem_bytes);

// Number of SMs of the current device.
int sem_num_sms();

// Per-class coefficient blocks of the plane-per-lane kernel (layout
// plane_layout(n) in sem_internal.h), computed in FP64, stored in FP32.
void launch_plane_coeffs(const SemGeom& g, const SemBasis& b, const double* dcoef, float* plane, cudaStream_t s);
// y += Hhat~ x with the plane-per-lane kernel (FP32, plane_supported(n));
// same contract as launch_tpt_apply.
void launch_plane_apply(const SemGeom& g, const SemClassTables<float>& t, const float* x, float* y,
                        double* partials, PcgState* st, cudaStream_t s);
// y += Hhat~ x with the k-slab kernel (FP32, slab_supported(n), class blocks of
// plane_layout(n)); same contract as launch_tpt_apply.
void launch_slab_apply(const SemGeom& g, const SemClassTables<float>& t, const float* x, float* y,
                       double* partials, PcgState* st, cudaStream_t s);

// Degrees served by the pencil kernel (sem_apply_pencil.cu): 5 <= n <= 8.
bool pencil_supported(int n);
// y += Hhat~ x with the pencil kernel (class blocks of plane_layout(n));
// same contract as launch_tpt_apply.
void launch_pencil_apply(const SemGeom& g, const SemClassTables<float>& t, const float* x, float* y,
                         double* partials, PcgState* st, cudaStream_t s);

// Degrees served by the row kernel (sem_apply_row.cu).
inline bool row_supported(int n) { return n >= 2 && n <= 8; }
// Most row segments one launch takes (bounded by the partial sums of the dot product).
constexpr long long kRowMaxUnits = 1LL << 17;
// Whether the row kernel can take this mesh and these vectors: a supported
// degree, at most kRowMaxUnits segments, and x, y at the same address modulo
// 16 bytes (its bulk copies keep that alignment).
bool row_usable(const SemGeom& g, const float* x, const float* y);
// y += Hhat~ x with the row kernel; same contract as launch_tpt_apply.
void launch_row_apply(const SemGeom& g, const SemBasis& b, const SemClassTables<float>& t, const float* x, float* y,
                      double* partials, PcgState* st, cudaStream_t s);

// Per-class operator coefficient blocks (layout in sem_internal.h), computed in
// FP64 and stored in T.
template <typename T>
void launch_class_coeffs(const SemGeom& g, const SemBasis& b, const double* dcoef, const double* dinv, T* coef,
                         cudaStream_t s);
// soa[r * ncls + c] = coef[c * stride + r]: the class blocks transposed, so
// that threads of consecutive classes read one coefficient with one
// coalesced load (the thread-per-element kernel, n = 1).
template <typename T>
void launch_coef_soa(const SemGeom& g, const T* coef, T* soa, long long stride, cudaStream_t s);
// y += Hhat~ x with the FP32 thread-per-element kernel (elem_supported(n),
// transposed class blocks of plane_layout(n)); same contract as launch_tpt_apply.
void launch_elem_apply(const SemGeom& g, const SemClassTables<float>& t, const float* x, float* y,
                       double* partials, PcgState* st, cudaStream_t s);

// y = Hhat~ x on the skeleton (transformed space); y must be zero on entry.
// If st != nullptr: also x^T y -> st->pq and alpha = rho / pq (CG step).
// cfg: optional kernel choice (nullptr or kind kApplyAuto: the built-in
// choice sem_apply_default_kind).
template <typename T>
void launch_tpt_apply(const SemGeom& g, const SemBasis& b, const SemClassTables<T>& t, const T* x, T* y,
                      double* partials, PcgState* st, cudaStream_t s, const ApplyConfig* cfg = nullptr);

void launch_class_tables(const SemGeom& g, const SemBasis& b, const double* ux_w, const double* uy_w,
                         const double* uz_w, double lambda, double* dcoef, double* dinv,
                         cudaStream_t s);

// diag of the assembled transformed condensed operator (atomics into diag, zeroed).
void launch_precond_diag(const SemGeom& g, const SemBasis& b, const SemClassTables<double>& t,
                         double* diag, cudaStream_t s);
// P = 1/diag on free entries, 0 on Dirichlet entries (diag in, P out; may alias).
void launch_invert_diag(const SemGeom& g, const double* diag, double* P, cudaStream_t s);

// Entity-wise skeleton transform with the n x n matrix A (device, row-major):
// faces U -> A U A^T, edges u -> A u, vertices copied.  in may alias out.
void launch_skel_transform(const SemGeom& g, const double* A, const double* in, double* out,
                           cudaStream_t s);

// Lumped-mass loads.  The assembled GLL mass at global node (gx, gy, gz) is
// mxs[gx] mys[gy] mzs[gz] (a product of 1D assembled masses).
// Skeleton: out[i] = mass * f at skeleton node i, 0 on Dirichlet entries.
void launch_load_skeleton(const SemGeom& g, const double* mxs, const double* mys, const double* mzs,
                          const double* f, double* out, cudaStream_t s);
// Interior cubes X[e][k][j][i] = mass * f at the element's interior nodes.
void launch_interior_load(const SemGeom& g, const double* mxs, const double* mys, const double* mzs,
                          const double* f, double* X, cudaStream_t s);

// Mode product along `axis` (0: i, 1: j, 2: k) of all interior cubes with the
// n x n matrix A in FP64: out[.. r ..] = sum_c A[r][c] in[.. c ..].  If
// grid != nullptr the result is written to the interior nodes of the full
// nodal field instead.
void launch_mode(const SemGeom& g, const double* A, int axis, const double* in, double* out,
                 double* grid, cudaStream_t s);
// The three mode products (A (x) A (x) A) of all interior cubes with the n x n
// matrix A: x[.. r ..] <- sum_c A[r][c] x[.. c ..] along i, then j, then k,
// in double-float arithmetic on the FP32 pipe (about 48 significant bits,
// each element's cube scaled by a power of two).  in: FP64 cubes (nelem n^3
// values, overwritten), tmp: scratch of the same size, eexp: nelem ints of
// scratch; the result goes to out (FP64 cubes), or, if grid != nullptr, to
// the interior nodes of the full nodal field.
void launch_mode3(const SemGeom& g, const double* A, double* in, double* tmp, int* eexp, double* out, double* grid,
                  cudaStream_t s);

// Condensed-load correction: Z = D^-1 Ft_I per element; out faces -= d k . Z.
void launch_condense_faces(const SemGeom& g, const SemBasis& b, const SemClassTables<double>& t,
                           const double* FtI, double* out, cudaStream_t s);

// Recovery: Z = D^-1 (Ft_I - H~_IB u~_B) per element (transformed interior).
void launch_recover_expand(const SemGeom& g, const SemBasis& b, const SemClassTables<double>& t,
                           const double* FtI, const double* uB, double* Z, cudaStream_t s);

void launch_pack(const SemGeom& g, const double* full, double* uB, cudaStream_t s);
// Writes skeleton values into the full field; zero_dirichlet writes 0 at
// domain-boundary nodes instead of the input value.
void launch_unpack(const SemGeom& g, const double* uB, double* full, int zero_dirichlet, cudaStream_t s);

// ---- CG vector kernels (T = double, or float for the inner solver) ----
// r = b - q (keep_x: q = A x0 on entry) else r = b and x = 0; z = P r; p = z;
// q = 0; rho = r.z, rr = r.r, rr0 = b.b, tol2 = rtol^2 rr0.
template <typename T>
void launch_pcg_init(long long nb, const T* b, T* r, T* p, T* q, T* x, const prec_t<T>* P, double* partials,
                     PcgState* st, double rtol, int maxit, int keep_x, cudaStream_t s);
// alpha from st: r -= alpha q; rho_new = r.P r, rr = r.r; convergence test.
// When it stops the CG, the iteration's x += alpha p is owed (st->xpend).
template <typename T>
void launch_pcg_update(long long nb, T* r, const T* q, const prec_t<T>* P, double* partials, PcgState* st,
                       cudaStream_t s);
// x += alpha p, then p = P r + beta p, q = 0.
template <typename T>
void launch_pcg_dir(long long nb, T* x, const T* r, T* p, T* q, const prec_t<T>* P, PcgState* st, cudaStream_t s);
// One-pass CG step (k_pcg_step: the update and the direction of one iteration
// with a grid barrier between them; cooperative launch, one CTA per SM).
// prepare_pcg_step sets the kernel's shared-memory limit (call outside graph
// capture) and reports whether the device can run it for vectors of nb.
template <typename T>
cudaError_t prepare_pcg_step(long long nb, bool* usable);
template <typename T>
cudaError_t launch_pcg_step(long long nb, T* x, T* r, T* p, T* q, const prec_t<T>* P, double* partials, PcgState* st,
                            cudaStream_t s);
// Applies an owed x += alpha p (no-op when none is owed; idempotent).
template <typename T>
void launch_pcg_flush(long long nb, T* x, const T* p, PcgState* st, cudaStream_t s);

// Iterative refinement: r = b - Ax and st->rr = r.r (FP64); out = (float)(in * scale);
// x += scale * c.
void launch_ir_residual(long long nb, const double* b, const double* Ax, double* r, double* partials,
                        PcgState* st, cudaStream_t s);
void launch_scale_to_f32(long long n, const double* in, double scale, float* out, cudaStream_t s);
void launch_ir_update(long long nb, double* x, const float* c, double scale, cudaStream_t s);
void launch_cast_f32(long long n, const double* in, float* out, cudaStream_t s);
// out = in rounded to the FP32 CG's preconditioner storage type (BF16, nearest even).
void launch_cast_prec32(long long n, const double* in, prec_t<float>* out, cudaStream_t s);
// Device-side refinement of a mixed-precision solve (one MixedCtl per
// problem): start after the FP64 residual r = b (st64) and the FP32 CG
// initialisation; one step per loop trip (gate, fold x32 into x, FP64
// operator q = A x through `gate`, residual and decision, rebase and
// direction of the FP32 CG), each kernel running only in its phase.
void launch_mixed_start(MixedCtl* ctl, const PcgState* st64, PcgState* st32, double rtol, double delta,
                        int max_refine, cudaStream_t s);
void launch_mixed_step(const SemGeom& g, const SemBasis& b, const SemClassTables<double>& tab, const ApplyConfig* op,
                       const double* rhs, double* x, double* q, double* r, float* x32, float* r32, float* p32,
                       float* q32, const prec_t<float>* P32, double* partials, MixedCtl* ctl, PcgState* st32,
                       PcgState* gate, cudaStream_t s);

int sem_vec_blocks();

// ---- adjoint support ----
// out = in / m (multiply = 0) or in * m (multiply = 1) at free nodes, 0 on the
// boundary; m the assembled lumped mass of the full nodal grid.
void launch_mass_divide(const SemGeom& g, const double* mxs, const double* mys, const double* mzs, const double* in,
                        double* out, int multiply, cudaStream_t s);
// E[e][0..3] = w_e^T K_k u_e on the reference element (K_0 = M(x)M(x)M, K_1 =
// M(x)M(x)K, K_2 = M(x)K(x)M, K_3 = K(x)M(x)M), E[e][4] = sum w w w w_e f_e.
void launch_element_forms(const SemGeom& g, const double* wgll, const double* K, const double* w, const double* u,
                          const double* f, double* E, cudaStream_t s);
// out[i] = dJ/dh_axis[i] from the element forms (device widths hx, hy, hz).
void launch_width_gradient(const SemGeom& g, int axis, const double* hx, const double* hy, const double* hz,
                           double lambda, const double* E, double* out, cudaStream_t s);
// *out = -sum_free w m u.
void launch_lambda_gradient(const SemGeom& g, const double* mxs, const double* mys, const double* mzs,
                            const double* w, const double* u, double* partials, double* out, unsigned int* counter,
                            cudaStream_t s);

#ifdef SEM_DEBUG
// Bounds records of the debug build, one per translation unit (SEM_DEBUG_TU in
// sem_device.cuh): each adds its count, keeps the first offending value and
// clears its record.
cudaError_t sem_debug_take_kernels(unsigned long long* count, long long* first);
cudaError_t sem_debug_take_apply(unsigned long long* count, long long* first);
cudaError_t sem_debug_take_plane(unsigned long long* count, long long* first);
cudaError_t sem_debug_take_slab(unsigned long long* count, long long* first);
cudaError_t sem_debug_take_elem(unsigned long long* count, long long* first);
cudaError_t sem_debug_take_row(unsigned long long* count, long long* first);
cudaError_t sem_debug_take_pencil(unsigned long long* count, long long* first);
cudaError_t sem_debug_take_compare(unsigned long long* count, long long* first);
#endif

// ---- the paper's comparison variants (sem_compare.cu): nodal skeleton, FP64, p <= 16
// Device state of the nodal-space CG of the comparison solvers.
struct CmpState {
  double rho, pq, rr, rr0, tol2, alpha, beta;
  int iter, done, maxit, pad;   // done: 1 converged, 2 breakdown, 3 maxit
  unsigned int counter[4];
};
constexpr int kCmpMaxP = 16;
// v += Hhat u (nodal): primary part, plus the TPC condensed part when condensed != 0.
void launch_tpc_apply(const SemGeom& g, const SemBasis& b, const SemClassTables<double>& t, const double* K,
                      const double* w, const double* A, const double* B, const double* u, double* v, int condensed,
                      cudaStream_t s);
// Dense condensed face-to-face matrix (6n^2 x 6n^2) of one width class.
void launch_mmc_build(const SemGeom& g, const SemBasis& b, const SemClassTables<double>& t, const double* A, int cls,
                      double* C, cudaStream_t s);
void launch_mmc_gather(const SemGeom& g, const int* elems, int count, const double* u, double* U, cudaStream_t s);
void launch_mmc_scatter(const SemGeom& g, const int* elems, int count, const double* Y, double* v, cudaStream_t s);
// diag += the assembled diagonal of the nodal condensed operator (cd: per-class scratch of ncls * 6n^2).
void launch_cmp_diag(const SemGeom& g, const SemBasis& b, const SemClassTables<double>& t, const double* K,
                     const double* w, const double* A, int ncls, double* cd, double* diag, cudaStream_t s);
void launch_cmp_init(long long nb, const double* b, double* x, double* r, const double* z, double* p, double* partials,
                     CmpState* st, double rtol, int maxit, cudaStream_t s);
void launch_cmp_pq(long long nb, const double* p, const double* q, double* partials, CmpState* st, cudaStream_t s);
void launch_cmp_xr(long long nb, double* x, double* r, const double* p, const double* q, double* partials,
                   CmpState* st, cudaStream_t s);
void launch_cmp_rz(long long nb, const double* r, const double* z, double* partials, CmpState* st, cudaStream_t s);
void launch_cmp_dir(long long nb, const double* z, double* p, double* q, const CmpState* st, cudaStream_t s);
void launch_cmp_diagmul(long long nb, const double* D, const double* r, double* z, const CmpState* st,
                        cudaStream_t s);

