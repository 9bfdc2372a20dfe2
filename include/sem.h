/*
 * sem.h -- C ABI of the GB300 (sm_103a) statically condensed spectral-element
 * Helmholtz solver.
 *
 * Problem (Sec. 3, Eq. helmholtz_equation):  lambda u - Laplace u = f on the box
 * [0, sum hx] x [0, sum hy] x [0, sum hz], lambda >= 0, homogeneous Dirichlet
 * boundary values, discretised by a Cartesian mesh of mx * my * mz hexahedral
 * spectral elements of degree p on Gauss-Lobatto-Legendre (GLL) nodes.  Element
 * (ex, ey, ez) has widths (hx[ex], hy[ey], hz[ez]).
 *
 * The library applies the statically condensed operator
 *     Hhat = H_BB - H_BI H_II^-1 H_IB          (Sec. 4, Eq. condensation_system)
 * element by element in the transformed, factorised form of Sec. 6 (Table 2 and
 * Eq. east_east_primary_part_transformed), inside a conjugate-gradient solver
 * with the block preconditioner that is diagonal in the transformed system
 * (solver "BT", Sec. 8), and recovers the interior unknowns by fast
 * diagonalisation (Algorithm 4).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * n = p - 1.  Global nodes form the grid Nx x Ny x Nz with Nx = mx p + 1 (etc.);
 * a "full nodal field" is a double array of Nx*Ny*Nz values, x fastest:
 * index gx + Nx (gy + Ny gz).
 *
 * A "skeleton vector" holds one value per node on element boundaries, packed
 * entity by entity (length N_B from sem_skeleton_size):
 *   1. x-faces (f, ey, ez), f in 0..mx: (mx+1) my mz faces, n*n values each,
 *      local (j, k) in 1..n, j fastest; node (f p, ey p + j, ez p + k)
 *   2. y-faces (ex, f, ez): mx (my+1) mz faces, local (i, k), i fastest
 *   3. z-faces (ex, ey, f): mx my (mz+1) faces, local (i, j), i fastest
 *   4. x-edges (ex, vy, vz): mx (my+1)(mz+1) edges, n values, local i
 *   5. y-edges (vx, ey, vz): (mx+1) my (mz+1) edges, local j
 *   6. z-edges (vx, vy, ez): (mx+1)(my+1) mz edges, local k
 *   7. vertices (vx, vy, vz): (mx+1)(my+1)(mz+1)
 * Within each block the first entity index is fastest.  Entities on the domain
 * boundary are present and held at zero: inputs there are ignored, outputs
 * there are written as zero.
 *
 * Spaces (sem_space): NODAL skeleton vectors are nodal values (or, for loads
 * and residuals, nodal load vectors).  TRANSFORMED vectors are those of Sec. 6:
 * with S_II from the generalised eigenproblem K_II V = M_II V Lambda,
 * V^T M_II V = I, S_II = V^T (eigenvalues ascending, each column of V scaled so
 * that its first entry is positive), a solution-like vector transforms as
 * u~ = T^-T u and a load-like vector as F~ = T F, where T applies S_II (x) S_II to
 * every face, S_II to every edge and 1 to every vertex.
 *
 * Memory and ownership: every vector argument is a caller-owned DEVICE pointer
 * (CUDA global memory of the device the context was created on, or managed
 * memory), aligned to its entry size (8 bytes, 4 for the FP32 vectors), unless
 * the name says host.  Every entry point checks this of each vector before any
 * launch (sem_check_vector) and returns SEM_EINVAL otherwise; the length
 * cannot be checked and is the caller's duty.  The library never frees caller
 * memory.  A context owns its precomputed tables and solver scratch on the
 * device it was created on.  A context is not thread-safe: use one context per
 * host thread.
 *
 * Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 * Operator, load and recovery calls are asynchronous on that stream.  sem_solve
 * returns after the solution is written (it synchronises to read its
 * convergence state).
 *
 * Errors: no exception crosses the ABI.  Arguments are checked before any
 * launch (SEM_EINVAL); CUDA failures return SEM_ECUDA; sem_last_error() gives
 * a human-readable message for the calling thread's last failure.
 */
#ifndef SEM_H
#define SEM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sem_ctx sem_ctx;

typedef enum {
  SEM_OK = 0,
  SEM_EINVAL = 1,     /* invalid argument (checked before any launch) */
  SEM_ENOMEM = 2,     /* device or host allocation failed */
  SEM_ECUDA = 3,      /* a CUDA call or kernel launch failed */
  SEM_ENOCONV = 4,    /* solver hit maxit; the best iterate is still written */
  SEM_EBREAKDOWN = 5, /* CG breakdown: p^T A p <= 0 or not finite (e.g. NaN input) */
  SEM_ENOTSUP = 6     /* valid request the library does not serve (N_B >= 2^31; batched scheme-0 mixed solves) */
} sem_status;

typedef enum { SEM_SPACE_NODAL = 0, SEM_SPACE_TRANSFORMED = 1 } sem_space;

typedef enum {
  SEM_PREC_FP64 = 0,  /* FP64 everywhere */
  SEM_PREC_MIXED = 1  /* FP32 inner CG inside FP64 iterative refinement */
} sem_precision;

/* Solver options.  Fill with sem_default_opts before changing fields. */
typedef struct {
  double rtol;        /* stop when ||r||_2 <= rtol ||b||_2 in the transformed
                         condensed space, b the condensed load (= ||r_0||_2 for a
                         zero start) (default 1e-10) */
  int maxit;          /* CG iteration cap, all refinement steps together (default 50000) */
  int precision;      /* sem_precision (default SEM_PREC_FP64) */
  int check_every;    /* CG iterations per device-side batch between host
                         convergence checks (default 16) */
  double inner_rtol;  /* MIXED scheme 0: residual reduction of each restarted FP32 inner
                         solve (default 1e-4) */
  int max_refine;     /* MIXED: cap on FP64 refinement steps (default 40) */
  int mixed_scheme;   /* MIXED: 1 = one FP32 CG kept across refinement steps, whose
                         residual is replaced by the FP64 residual at each step
                         ("reliable updates", default); 0 = the FP32 CG restarts from
                         zero at every refinement step (classical refinement) */
  double reliable_delta; /* MIXED scheme 1: a refinement step is taken when the FP32
                         recursive residual has fallen by this factor since the
                         previous step; 0 = automatic (default): 0.03 at p = 2,
                         0.01 otherwise (the fastest measured on GB300) */
  int deterministic;  /* FP64 operator: 1 (default) = the edge and vertex outputs (shared
                         by 4 and 8 elements) are summed in a fixed element order
                         through per-element scratch of nelem (12 (p-1) + 8) doubles,
                         allocated on first use, so FP64 solves (single or batched)
                         give the same bits and iteration counts on every run;
                         0 = atomic scatter-adds (arrival order).  Faces (two
                         elements, added onto zero) are exact either way.  The FP32
                         operators of MIXED solves always use atomics. */
  int onepass_step;   /* MIXED single solves: 1 (default) = the FP32 CG's update and
                         direction are one kernel that reads r, q, P, x, p and writes
                         r, x, p, q once per iteration (a grid barrier between the two
                         halves; cooperative launch, one CTA per SM holding its
                         range of z = P r in shared memory, the barrier's wait
                         bounded); 0 = two kernels (r, P read twice).  The one-pass
                         step is taken only where z fits (N_B up to 200 KB of FP32
                         per SM: 7.78e6 on 152 SMs); batched solves, larger N_B, or a
                         device or graph that cannot take the cooperative launch
                         run two kernels.  The step holds every SM: single mixed
                         solves of several contexts running concurrently on one
                         GPU should set 0 (otherwise their grids can wait on each
                         other until the barrier's bounded wait gives up and the
                         solve fails with SEM_EBREAKDOWN and a message naming it). */
} sem_opts;

/* Result of a solve. */
typedef struct {
  int iters;          /* CG iterations (sum over refinement steps for MIXED) */
  int refinements;    /* FP64 refinement steps (MIXED), 0 for FP64 */
  double rel_res;     /* final ||r||_2 / ||b||_2, FP64, transformed condensed space */
  double t_solve_s;   /* wall time of the solve, host clock, seconds */
} sem_info;

/* Fills *opts with the defaults listed above. */
void sem_default_opts(sem_opts* opts);

/* Creates a context (Sec. 3 problem statement; setup of Sec. 5-6 and the
 * diagonal of the transformed condensed operator, Sec. 8).
 *   p in [2, 32]; mx, my, mz >= 1; hx[mx], hy[my], hz[mz]: HOST arrays of
 *   positive finite element widths; lambda >= 0 and finite; opts may be NULL.
 * Computes on the host the 1D GLL basis, the generalised eigenpairs and the
 * transformed stiffness vectors, then on the device per element-width class
 * the metric coefficients (Eq. metriccoeffelement), D^-1 (Eq. hii_diagonal)
 * and the diagonal preconditioner.  Allocates all device scratch.  On success
 * *out owns everything; release it with sem_destroy.  Uses the current CUDA
 * device; synchronises before returning. */
sem_status sem_setup(sem_ctx** out, int p, int mx, int my, int mz,
                     const double* hx, const double* hy, const double* hz,
                     double lambda, const sem_opts* opts);

/* Changes lambda (the paper's time-step dependent Helmholtz parameter, Sec. 8)
 * and recomputes D^-1 and the preconditioner.  Synchronous. */
sem_status sem_set_lambda(sem_ctx* ctx, double lambda);

/* Replaces the solver options of an existing context (NULL = defaults). */
sem_status sem_set_opts(sem_ctx* ctx, const sem_opts* opts);

/* N_B, the packed skeleton length (see the layout above). */
sem_status sem_skeleton_size(const sem_ctx* ctx, long long* nb);

/* Number of global nodes Nx*Ny*Nz of a full nodal field. */
sem_status sem_grid_size(const sem_ctx* ctx, long long* n_nodes);

/* Global node coordinates along each axis, HOST arrays of length Nx, Ny, Nz
 * (element offsets plus the GLL points mapped to each element). */
sem_status sem_node_coords(const sem_ctx* ctx, double* x, double* y, double* z);

/* 1D basis used by the context, HOST arrays: gll_x[p+1], gll_w[p+1],
 * lambda_1d[n] (ascending) and V[n*n] row-major (V[r*n + c] = entry r of
 * eigenvector c), canonical signs as described above.  Any pointer may be NULL. */
sem_status sem_get_basis(const sem_ctx* ctx, double* gll_x, double* gll_w,
                         double* lambda_1d, double* V);

/* v_B = Rhat Hhat Rhat^T u_B on the skeleton (Sec. 4 operator, assembled).
 * NODAL: u and v are nodal skeleton vectors (v is a load vector).
 * TRANSFORMED: v~ = T Hhat T^T u~, the operator the CG iterates on.
 * uB, vB: device, length N_B, must not overlap.  Asynchronous on stream. */
sem_status sem_apply_condensed(sem_ctx* ctx, const double* uB, double* vB,
                               sem_space space, void* stream);

/* The transformed condensed operator in FP32 (the operator of the mixed-
 * precision inner solver): v~ = T Hhat T^T u~ with FP32 tables and
 * arithmetic.  uB, vB: device float arrays of length N_B, not overlapping.
 * Prepares the FP32 tables on first use.  Asynchronous on stream. */
sem_status sem_apply_condensed_f32(sem_ctx* ctx, const float* uB, float* vB, void* stream);

/* Condensed load fhat = sum_e Rhat_e (F_B - H_BI H_II^-1 F_I) (Algorithm 1,
 * first loop; Algorithm 4 in the TRANSFORMED space), with F_e the GLL-quadrature
 * load of the nodal field f: F_e = (h1 h2 h3 / 8) (w (x) w (x) w) o f_e.
 * f: device full nodal field; fB: device skeleton vector.  Asynchronous.
 * The interior transforms (S (x) S (x) S on every element) are computed in
 * double-float arithmetic on the FP32 pipe: about 48 significant bits, each
 * element's values scaled by a power of two first, so the result stays
 * within about 1e-13 of FP64 arithmetic relative to its norm. */
sem_status sem_condense_rhs(sem_ctx* ctx, const double* f, double* fB,
                            sem_space space, void* stream);

/* Diagonal of the assembled transformed condensed operator T Hhat T^T (the
 * BT preconditioner is its inverse, Sec. 8).  diag: device skeleton vector;
 * Dirichlet entries are written as zero.  Asynchronous. */
sem_status sem_precond_diag(sem_ctx* ctx, double* diag, void* stream);

/* Interior recovery (Algorithm 4, second loop): u_I = H_II^-1 (F_I - H_IB u_B)
 * per element, back-transformed, written with the skeleton values into the
 * full nodal field u.  uB is a skeleton solution in `space`.  f, u: device full
 * nodal fields (u is fully overwritten, Dirichlet nodes with 0).  Asynchronous.
 * The back-transform of the interiors is computed in double-float arithmetic
 * like the load's (sem_condense_rhs). */
sem_status sem_recover_interior(sem_ctx* ctx, const double* f, const double* uB,
                                sem_space space, double* u, void* stream);

/* Full solve (Algorithm 4): condense the load, CG with the BT preconditioner
 * to opts.rtol, recover the interior.  With opts.precision = SEM_PREC_MIXED the
 * CG runs in FP32 (FP32 operator and vectors, the preconditioner stored in
 * BF16) inside FP64
 * iterative refinement: every refinement step adds the FP32 correction to the
 * FP64 iterate x and recomputes the residual r = b - A x with the FP64
 * operator and FP64 dot products (see opts.mixed_scheme); the stopping rule
 * is that FP64 residual.  f, u: device full nodal fields; u0:
 * optional device skeleton start vector in NODAL space (NULL = 0); info may be
 * NULL.  Returns SEM_ENOCONV / SEM_EBREAKDOWN with u still written. */
sem_status sem_solve(sem_ctx* ctx, const double* f, double* u, const double* u0,
                     sem_info* info, void* stream);

/* sem_solve on HOST arrays f_host, u_host (full nodal fields): copies f to the
 * device, solves, copies u back, all on `stream`; returns when u_host is
 * written.  Pinned host memory gives the fastest copies.  The two device
 * fields it copies through are allocated on the first call and kept by the
 * context (freed by sem_destroy); SEM_ENOMEM if they cannot be allocated. */
sem_status sem_solve_host(sem_ctx* ctx, const double* f_host, double* u_host,
                          sem_info* info, void* stream);

/* Transform of a skeleton vector between spaces (see "Spaces" above):
 * kind 0: u~ = T^-T u (solution, nodal -> transformed)
 * kind 1: u  = T^T u~ (solution, transformed -> nodal)
 * kind 2: F~ = T F    (load, nodal -> transformed)
 * kind 3: F  = T^-1 F~ (load, transformed -> nodal)
 * in, out: device, length N_B, may alias.  Asynchronous. */
sem_status sem_transform_skeleton(sem_ctx* ctx, const double* in, double* out,
                                  int kind, void* stream);

/* Skeleton <-> full nodal field: pack gathers the skeleton nodes of u_full into
 * uB; unpack writes uB into the skeleton nodes of u_full (other nodes are left
 * untouched).  Device pointers.  Asynchronous. */
sem_status sem_pack_skeleton(sem_ctx* ctx, const double* u_full, double* uB, void* stream);
sem_status sem_unpack_skeleton(sem_ctx* ctx, const double* uB, double* u_full, void* stream);

/* sem_condense_rhs without any memory allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory at the time of the call -- an application
 * whose own pool allocator has reserved the device memory up front (where a
 * cudaMalloc fails or eats into the pool), or a latency-bound loop that must
 * not take the device-wide synchronisation that cudaFree (and at times
 * cudaMalloc) makes.  sem_condense_rhs allocates its element-interior scratch
 * with cudaMalloc on first use; this variant calls no cudaMalloc, cudaFree or
 * other allocating routine and instead uses a fixed scratch array compiled
 * into the library (12 MiB, held by every GPU that loads the library until
 * the process exits).
 *   ctx, f, fB, space, stream: as for sem_condense_rhs (same result to
 *   about 1e-13: this variant's interior transforms run in FP64, the fixed
 *   array having no room for the per-element scale exponents of the
 *   double-float form).
 *   Limit: elements * (p-1)^3 <= 524288 (e.g. p = 8 on 8^3 elements, p = 4 on
 *   16^3); larger meshes are rejected with SEM_EINVAL and a message.
 * The first call on each device looks up the scratch array's device address;
 * make that first call before any stream capture.  All calls share the one
 * array: calls that overlap on the GPU (different streams, or concurrent host
 * threads) race on it and must be serialised by the caller.  Nothing needs to
 * be cleared between calls.  Asynchronous on `stream`. */
sem_status sem_condense_rhs_noalloc(sem_ctx* ctx, const double* f, double* fB,
                                    sem_space space, void* stream);

/* Adjoint solve for gradients of a solve: w = A^-1 g, A the assembled
 * (uncondensed) Helmholtz operator on the free nodes and g a nodal load vector
 * (for J(u), g = dJ/du).  A is symmetric, so this is the same condensed solve
 * as sem_solve with the load g in place of (lumped mass) o f.  g, w: device
 * full nodal fields; boundary entries of g are ignored and w is 0 there.
 * Uses the context's options (precision, rtol).  Allocates its buffers on
 * first use. */
sem_status sem_solve_adjoint(sem_ctx* ctx, const double* g, double* w, sem_info* info, void* stream);

/* Gradients of J(u(f, lambda, h)) from the adjoint w of a solve u (u =
 * sem_solve(f), w = sem_solve_adjoint(dJ/du)):
 *   df        = M w                          (device full field; 0 on the boundary)
 *   *dlambda  = -w^T M u                     (M: assembled lumped mass, dA/dlambda)
 *   dh*[i]    = sum over the elements of slab i of
 *               -sum_k (dd_k/dh) w_e^T K_k u_e + (dJ_e/dh) sum_abc w_a w_b w_c (w f)_e,
 * with d = J (lambda, 4/h1^2, 4/h2^2, 4/h3^2), J = h1 h2 h3 / 8
 * (Eq. metriccoeffelement) and K_k the Kronecker terms of Eq. helmholtz_operator.
 * w, u, f, df: device full fields.  dlambda, dhx[mx], dhy[my], dhz[mz]: HOST
 * outputs (may be NULL).  Synchronous. */
sem_status sem_gradients(sem_ctx* ctx, const double* w, const double* u, const double* f, double* df,
                         double* dlambda, double* dhx, double* dhy, double* dhz, void* stream);

/* Operator kernel variants.  All compute the same transformed condensed
 * operator (Sec. 6, Table 2); they differ only in how the elements' work is
 * mapped onto the GPU.  The paper has no counterpart: this is a performance
 * choice of this library.
 *   SEM_KERNEL_AUTO      the built-in choice for the degree and precision
 *   SEM_KERNEL_CTA_TILE  a CTA works on a tile of epb elements, the n^3
 *                        eigenspace cube in slabs of ks planes (any degree)
 *   SEM_KERNEL_WARP      one warp per element (FP32, 3 <= n <= 7)
 *   SEM_KERNEL_PLANE     one lane per plane of the cube: a group of 4 or 8
 *                        lanes per element for 2 <= n <= 8, one warp per
 *                        element (two lanes per plane, each a half row) for
 *                        9 <= n <= 15 (FP32)
 *   SEM_KERNEL_ELEMENT   one thread per element (p = 2; FP32 also p = 3, 4)
 *   SEM_KERNEL_SLAB      a CTA works on one element and a slab of 8 planes k
 *                        of its eigenspace cube at a time (FP32,
 *                        16 <= n <= 31)
 *   SEM_KERNEL_ROW       a CTA works on a segment of up to 32 consecutive
 *                        elements of one x-row: warp w takes plane w of every
 *                        element's cube, lane l element l; the segment's
 *                        skeleton ranges move by bulk copies and bulk
 *                        reduce-adds (FP32, 2 <= n <= 8; vectors whose
 *                        addresses differ by a multiple of 16 bytes, else it
 *                        runs as PLANE)
 *   SEM_KERNEL_PENCIL    a CTA holds 256 / n^2 elements: one thread per
 *                        x-pencil (j, k) forms D^-1 x along i and the x-face
 *                        outputs, then one thread per cube column (i, m)
 *                        the y- and z-face outputs and the edge and vertex
 *                        outputs (FP32, 5 <= n <= 8)
 * where n = p - 1.  SEM_KERNEL_AUTO resolves, in FP64, to ELEMENT at p = 2
 * and CTA_TILE otherwise; in FP32 to ELEMENT at p <= 3, PLANE for
 * 4 <= p <= 16 and SLAB for 17 <= p <= 32 (the fastest measured on GB300;
 * sem_autotune ranks the alternatives for a given mesh). */
enum {
  SEM_KERNEL_AUTO = 0,
  SEM_KERNEL_CTA_TILE = 1,
  SEM_KERNEL_WARP = 2,
  SEM_KERNEL_PLANE = 3,
  SEM_KERNEL_ELEMENT = 4,
  SEM_KERNEL_SLAB = 5,
  SEM_KERNEL_ROW = 6,
  SEM_KERNEL_PENCIL = 7
};

/* Selects the operator kernel of one precision: SEM_PREC_FP64 (the FP64
 * operator of FP64 solves, of the refinement residuals and of
 * sem_apply_condensed) or SEM_PREC_MIXED (the FP32 operator of the inner CG
 * and of sem_apply_condensed_f32).  epb (1..64) and ks (1..n) are used by
 * SEM_KERNEL_CTA_TILE only.  Applies to every later call on this context;
 * batches created earlier keep the kernel they captured.  Returns SEM_EINVAL
 * if the variant does not exist for this degree and precision, or the tile
 * does not fit in shared memory. */
sem_status sem_set_operator_kernel(sem_ctx* ctx, int precision, int kind, int epb, int ks);
/* The kernel in use for one precision, SEM_KERNEL_AUTO resolved: *kind, and
 * for a CTA tile *epb, *ks (else 0; epb, ks may be NULL). */
sem_status sem_get_operator_kernel(const sem_ctx* ctx, int precision, int* kind, int* epb, int* ks);
/* The check every entry point makes of a vector argument, without any launch:
 * SEM_OK if p is not null, is a multiple of elem_bytes (4 or 8) and points to
 * device memory of the context's device or to managed memory; else SEM_EINVAL
 * with the reason in sem_last_error(). */
sem_status sem_check_vector(const sem_ctx* ctx, const void* p, int elem_bytes);
/* Bounds record of a debug build (the library compiled with SEM_DEBUG, see
 * paper_1601_08179_gb300/build.py): every kernel checks each skeleton entity
 * offset it forms (and each class index) against its range before any access,
 * counts the failures, keeps the first offending value and skips the entity.
 * sem_debug_oob synchronises the device, returns the count since the last call
 * in *count and the first value in *first (-1 if none), and clears the record.
 * sem_debug_limit_skeleton lowers the bound the checks of this context's later
 * launches compare against (0 <= bound <= N_B; N_B restores it), so that a
 * test can show an offending offset is caught while every access stays inside
 * the real vectors.  Both return SEM_ENOTSUP in release builds. */
sem_status sem_debug_oob(long long* count, long long* first);
sem_status sem_debug_limit_skeleton(sem_ctx* ctx, long long bound);
/* Failure check of the one-pass CG step's grid barrier (debug builds): runs
 * one step of the FP32 CG on zeroed vectors with the barrier's arrival count
 * preset past the grid size, so that no CTA ever completes the barrier; each
 * CTA's bounded wait (about a second) runs out, and the step stops the CG.
 * Returns the step's record: *bar_fail (1 when a wait ran out) and *done (2:
 * stopped as a breakdown).  The context stays usable (its FP32 CG record is
 * cleared afterwards).  SEM_ENOTSUP in release builds or where the device
 * cannot take the cooperative launch. */
sem_status sem_debug_cg_step_timeout(sem_ctx* ctx, int* bar_fail, int* done);
/* Autotuner: times the operator kernel for this context's degree, mesh and
 * precision (FP32 when opts.precision is MIXED, else FP64) over the variants
 * that exist for it and a set of CTA-tile shapes (elements per CTA,
 * eigenspace slab depth), keeps the fastest (the built-in choice included)
 * for all later applications and solves, and caches the choice per
 * (p, mx, my, mz, precision) for the process.  *ms_default / *ms_best (may be
 * NULL): milliseconds per application of the built-in and the chosen
 * configuration.  Synchronous. */
sem_status sem_autotune(sem_ctx* ctx, double* ms_default, double* ms_best);

/* Batched solves (independent problems of any degree and mesh size).
 * sem_batch_create captures, for `count` distinct contexts with device
 * fields f[i] (input) and u[i] (output), ONE CUDA graph: a prologue that
 * condenses every load and initialises every CG (one graph branch per
 * problem), a device-side `while` loop whose body runs opts.check_every CG
 * iterations of every problem in parallel branches followed by a one-thread
 * kernel that ends the loop once no problem is still running (bounded by the
 * largest maxit), and an epilogue that recovers every interior.  Converged
 * problems' kernels exit at once.  A context may be FP64 or mixed precision
 * with reliable updates (opts.mixed_scheme 1; scheme 0 is SEM_ENOTSUP): a
 * mixed problem's loop body first runs its FP64 refinement step when one is
 * due (its FP32 CG stops itself once its residual has fallen by
 * opts.reliable_delta), all decided on the device, then FP32 CG iterations;
 * infos[i].refinements and sem_refine_history report its steps.  The graph bakes in the context and field
 * pointers; create a new batch when they change.  sem_batch_solve launches the
 * graph once on `stream` and fills infos[count] (may be NULL); it returns
 * SEM_ENOCONV or SEM_EBREAKDOWN if any problem failed (all u[i] are written).
 * The contexts must not be used concurrently while the batch runs.
 * sem_solve_batch = create + solve + destroy. */
typedef struct sem_batch sem_batch;
sem_status sem_batch_create(sem_ctx* const* ctxs, int count, const double* const* f, double* const* u,
                            sem_batch** out);
sem_status sem_batch_solve(sem_batch* batch, sem_info* infos, void* stream);
void sem_batch_destroy(sem_batch* batch);
sem_status sem_solve_batch(sem_ctx* const* ctxs, int count, const double* const* f, double* const* u,
                           sem_info* infos, void* stream);

/* The paper's comparison variants (Sec. 5 and Sec. 8), on the NODAL skeleton
 * in FP64.  They exist to measure the transformed operator and solver this
 * library is built on against the alternatives the paper compares them with.
 * Operators (sem_apply_condensed_variant: vB = Hhat uB, the same operator as
 * sem_apply_condensed in SEM_SPACE_NODAL, computed another way):
 *   SEM_OP_TPT  the transformed operator (Table 2) between the skeleton
 *               transforms: what sem_apply_condensed(NODAL) does
 *   SEM_OP_TPC  Algorithm 3 with Table 1: the nodal primary part
 *               (Eq. east_east_primary_part, 12 n^3 multiplications per
 *               element) and the condensed part through the interior
 *               eigenspace, the faces mapped in and out with V^T M_II and
 *               M_II V inside the element loop (37 n^3); p <= 16
 *   SEM_OP_MMC  Algorithm 2: the nodal primary part and the condensed part as
 *               a dense 6n^2 x 6n^2 face-to-face matrix per width class,
 *               applied to all elements of a class with one DGEMM (36 n^4);
 *               built on first use (O(n^7) per class); p <= 16, at most
 *               8 GiB of matrices (else SEM_ENOTSUP)
 * Preconditioners of sem_solve_variant (CG on the nodal condensed system,
 * stopping at ||r|| <= opts.rtol ||b||, at most opts.maxit iterations):
 *   SEM_PC_NONE   unpreconditioned (the paper's UC with TPC)
 *   SEM_PC_DIAG   inverse diagonal of the nodal condensed operator (DC)
 *   SEM_PC_BLOCK  exact inverse of the face, edge and vertex self blocks (BC),
 *                 applied in tensor form: transform, the inverse diagonal of
 *                 the transformed operator, transform back (the blocks are
 *                 diagonal in the transformed system)
 * sem_diag_nodal writes the assembled diagonal of the nodal condensed
 * operator (0 at Dirichlet entries).  Vectors: device, N_B (uB, vB, diag) or
 * the full nodal grid (f, u).  sem_apply_condensed_variant and sem_diag_nodal
 * are asynchronous; sem_solve_variant synchronises to read its stopping test
 * after every iteration and fills info (iters, rel_res, t_solve_s). */
enum { SEM_OP_TPT = 0, SEM_OP_TPC = 1, SEM_OP_MMC = 2 };
enum { SEM_PC_NONE = 0, SEM_PC_DIAG = 1, SEM_PC_BLOCK = 2 };
sem_status sem_apply_condensed_variant(sem_ctx* ctx, int op, const double* uB, double* vB, void* stream);
sem_status sem_diag_nodal(sem_ctx* ctx, double* diag, void* stream);
sem_status sem_solve_variant(sem_ctx* ctx, int op, int pc, const double* f, double* u, sem_info* info, void* stream);

/* Residual history of the last MIXED solve: rel_res[k] = ||b - A x_k|| / ||b||
 * (FP64, transformed condensed space) before refinement step k and after the
 * last one; *count = number of entries (up to max_refine + 1).  HOST array of
 * `capacity` entries; at most `capacity` are written. */
sem_status sem_refine_history(const sem_ctx* ctx, double* rel_res, int capacity, int* count);

/* Kernel timing inside sem_solve.  While enabled, every launch of the condensed
 * operator kernel inside the solver's CG iteration is bracketed by CUDA events
 * on the stream it runs on; sem_profile_read returns the summed device time
 * (milliseconds) and the number of timed launches since the last reset.
 * Enabling or disabling rebuilds the captured iteration graph. */
sem_status sem_profile_enable(sem_ctx* ctx, int enable);
sem_status sem_profile_read(sem_ctx* ctx, double* apply_ms, long long* apply_launches, int reset);

/* Number of kernel launches this library has issued in this process (graph
 * launches count each kernel node).  Monotone. */
long long sem_launch_count(void);

/* Releases every device and host resource of the context (NULL is a no-op). */
void sem_destroy(sem_ctx* ctx);

/* Static description of a status code. */
const char* sem_status_string(sem_status s);

/* Message of the calling thread's last failure ("" if none). */
const char* sem_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SEM_H */
