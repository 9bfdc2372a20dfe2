// C ABI of the condensed spectral-element Helmholtz library (include/sem.h).
//
// The context owns: the 1D basis (host), per-width-class tables (device),
// transform matrices, the BT preconditioner, CG vectors and scratch.  The
// FP64 solve follows Algorithm 4 of the paper:
//   1. transformed condensed load  fhat~ = T F_B - H~_BI D^-1 F~_I
//   2. CG on Hhat~ with the diagonal (block-Jacobi) preconditioner, batches of
//      iterations captured in a CUDA graph; the convergence test runs on the
//      device and the host reads one small status record per batch;
//   3. interior recovery u_I = (V(x)V(x)V) D^-1 (F~_I - H~_IB u~_B) and the
//      nodal skeleton u_B = T^T u~_B.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <map>
#include <tuple>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sem.h"
#include "sem_internal.h"
#include "sem_kernels.cuh"

namespace {

thread_local std::string t_err;

sem_status fail(sem_status s, const std::string& msg) {
  t_err = msg;
  return s;
}

#define SEM_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t _e = (call);                                                             \
    if (_e != cudaSuccess)                                                               \
      return fail(SEM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e));       \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, count * sizeof(T));
}

}  // namespace

struct sem_ctx {
  int device = 0;
  SemGeom g{};
  SemHost1D h1;
  double lambda = 0.0;
  sem_opts opts{};
  std::vector<double> hx, hy, hz;
  std::vector<double> uxw, uyw, uzw;
  std::vector<int> clsx, clsy, clsz;
  std::vector<double> xc, yc, zc;      // node coordinates per axis

  int* d_cls = nullptr;                // [mx + my + mz]
  double* d_uw = nullptr;              // [ux + uy + uz] distinct widths
  double* d_dcoef = nullptr;
  double* d_dinv = nullptr;
  double* d_coef = nullptr;            // per-class operator coefficient blocks (FP64)
  float* d_coef_f = nullptr;           // the same in FP32 (mixed precision)
  float* d_plane = nullptr;            // class blocks of the plane-per-lane FP32 kernel
  double* d_coef_soa = nullptr;        // n = 1: the class blocks transposed (FP64, FP32)
  float* d_coef_soa_f = nullptr;
  float* d_plane_soa = nullptr;        // n = 2, 3: the plane blocks transposed
  double* d_hf = nullptr;              // device copies of sem_solve_host's load and solution (first use)
  double* d_hu = nullptr;
  double* d_mats = nullptr;            // 4 n*n: S_II, V, V^T M_II, M_II V
  double* d_mass = nullptr;            // [Nx + Ny + Nz] assembled 1D lumped masses
  double* d_h = nullptr;               // [mx + my + mz] element widths
  double* d_K = nullptr;               // (p+1)^2 stiffness, [p+1] GLL weights
  double* d_full = nullptr;            // full-field scratch (adjoint right-hand side)
  double* d_E = nullptr;               // [n_e][5] element bilinear forms (gradients)
  double* d_grad = nullptr;            // [1 + mx + my + mz] gradient outputs
  double* d_P = nullptr;               // BT preconditioner (inverse diagonal)
  double *d_x = nullptr, *d_r = nullptr, *d_p = nullptr, *d_q = nullptr, *d_b = nullptr;
  double *d_t1 = nullptr, *d_t2 = nullptr;
  double *d_c0 = nullptr, *d_c1 = nullptr, *d_FtI = nullptr;   // interior cubes
  int* d_cexp = nullptr;               // per-element scale exponents of the mode products
  double* d_partials = nullptr;
  PcgState* d_st = nullptr;
  PcgState* h_st = nullptr;            // pinned
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_iters = 0;
  bool graph_prof = false;
  bool prof = false;                   // time operator launches inside the CG graph
  std::vector<cudaEvent_t> pev;        // 2 per captured iteration
  double prof_ms = 0.0;
  long long prof_count = 0;
  SemClassTables<double> tab{};

  // mixed precision (FP32 inner CG), allocated on first use
  float *d_dcoef_f = nullptr, *d_dinv_f = nullptr;
  prec_t<float>* d_P32 = nullptr;     // the FP32 CG's BT preconditioner (BF16)
  float *d_b32 = nullptr, *d_x32 = nullptr, *d_r32 = nullptr, *d_p32 = nullptr, *d_q32 = nullptr;
  PcgState* d_st32 = nullptr;
  MixedCtl* d_ctl = nullptr;           // device-side refinement control (graph-replayed mixed solves)
  MixedCtl h_ctl{};                    // host copy of it
  cudaGraphExec_t graph32m = nullptr;  // one loop trip of the reliable-update mixed solve (or the whole loop)
  int* d_trips = nullptr;              // trips of the device-side CG loops
  double* d_ev = nullptr;              // per-element edge/vertex shares (opts.deterministic)
  bool step_ok = false;                // the device runs the one-pass FP32 CG step (cooperative launch)
  bool step_failed = false;            // a graph with it could not be built: two-pass step from then on
  bool graph_loop = false, graph32m_loop = false;   // the graph holds the whole loop (a while node)
  long long graph_per_trip = 0, graph32m_per_trip = 0;
  int graph_cap = 0, graph32m_cap = 0;
  int graph32m_iters = 0;
  bool graph32m_prof = false;
  long long graph32m_launches = 0;
  PcgState* d_stg = nullptr;           // gate of the FP64 operator in those solves
  SemClassTables<float> tab_f{};
  cudaGraphExec_t graph32 = nullptr;
  int graph32_iters = 0;
  long long graph32_launches = 0;
  bool graph32_prof = false;
  std::vector<cudaEvent_t> pev32;
  std::vector<double> refine_hist;     // ||b - A x_k|| / ||b|| after each refinement step
  ApplyConfig op64{}, op32{};           // operator kernel per precision (kind kApplyAuto: built-in)

  // the paper's comparison variants (nodal skeleton, FP64), allocated on first use
  double* d_cmpK = nullptr;            // (p+1)^2 stiffness, then the (p+1) GLL weights
  double* d_cmp = nullptr;             // skeleton vectors of the nodal CG: b, x, r, p, q, z, tmp
  CmpState* d_cst = nullptr;
  CmpState h_cst{};
  double* d_cdiag = nullptr;           // per-class condensed face diagonals
  double* d_Pdc = nullptr;             // inverse diagonal of the nodal condensed operator (DC)
  double* d_mmc = nullptr;             // per-class dense condensed face matrices (MMC)
  int* d_cls_elems = nullptr;          // elements grouped by width class
  std::vector<long long> cls_start;
  std::vector<int> cls_count;
  double *d_mmcU = nullptr, *d_mmcY = nullptr;
  cublasHandle_t cublas = nullptr;

  const double* mat(int k) const { return d_mats + (size_t)k * g.n * g.n; }
};

namespace {

constexpr size_t kPartials = 1 << 17;

void build_classes(const std::vector<double>& h, std::vector<double>* uw, std::vector<int>* cls) {
  std::map<double, int> seen;
  cls->resize(h.size());
  uw->clear();
  for (size_t i = 0; i < h.size(); ++i) {
    auto it = seen.find(h[i]);
    if (it == seen.end()) {
      int id = (int)uw->size();
      seen[h[i]] = id;
      uw->push_back(h[i]);
      (*cls)[i] = id;
    } else {
      (*cls)[i] = it->second;
    }
  }
}

// 1D assembled lumped mass: m[e p + a] += (h_e / 2) w_a; node coordinates.
void axis_mass_coords(int p, const std::vector<double>& h, const std::vector<double>& xg,
                      const std::vector<double>& w, std::vector<double>* m, std::vector<double>* x) {
  const size_t N = h.size() * p + 1;
  m->assign(N, 0.0);
  x->assign(N, 0.0);
  double X0 = 0.0;
  for (size_t e = 0; e < h.size(); ++e) {
    for (int a = 0; a <= p; ++a) {
      (*m)[e * p + a] += 0.5 * h[e] * w[a];
      if (a < p) (*x)[e * p + a] = X0 + 0.5 * h[e] * (xg[a] + 1.0);
    }
    X0 += h[e];
  }
  (*x)[N - 1] = X0;
}

bool valid_widths(const double* h, int m) {
  if (h == nullptr) return false;
  for (int i = 0; i < m; ++i)
    if (!(h[i] > 0.0) || !std::isfinite(h[i])) return false;
  return true;
}

sem_status cast_tables_f32(sem_ctx* c, cudaStream_t s);

sem_status compute_tables(sem_ctx* c, cudaStream_t s) {
  const SemGeom& g = c->g;
  launch_class_tables(g, c->h1.basis, c->d_uw, c->d_uw + g.ux, c->d_uw + g.ux + g.uy, c->lambda, c->d_dcoef,
                      c->d_dinv, s);
  launch_class_coeffs<double>(g, c->h1.basis, c->d_dcoef, c->d_dinv, c->d_coef, s);
  if (c->d_coef_soa != nullptr) launch_coef_soa<double>(g, c->d_coef, c->d_coef_soa, coef_offsets(1).stride, s);
  SEM_CUDA(cudaGetLastError());
  SEM_CUDA(cudaMemsetAsync(c->d_t1, 0, sizeof(double) * g.nb, s));
  launch_precond_diag(g, c->h1.basis, c->tab, c->d_t1, s);
  launch_invert_diag(g, c->d_t1, c->d_P, s);
  SEM_CUDA(cudaGetLastError());
  if (c->d_st32 != nullptr) return cast_tables_f32(c, s);
  return SEM_OK;
}

sem_status cast_tables_f32(sem_ctx* c, cudaStream_t s) {
  const SemGeom& g = c->g;
  const long long ncls = (long long)g.ux * g.uy * g.uz;
  launch_cast_f32(ncls * 4, c->d_dcoef, c->d_dcoef_f, s);
  launch_cast_f32(ncls * (long long)g.n * g.n * g.n, c->d_dinv, c->d_dinv_f, s);
  launch_class_coeffs<float>(g, c->h1.basis, c->d_dcoef, c->d_dinv, c->d_coef_f, s);
  if (c->d_coef_soa_f != nullptr) launch_coef_soa<float>(g, c->d_coef_f, c->d_coef_soa_f, coef_offsets(1).stride, s);
  if (c->d_plane != nullptr) launch_plane_coeffs(g, c->h1.basis, c->d_dcoef, c->d_plane, s);
  if (c->d_plane_soa != nullptr) launch_coef_soa<float>(g, c->d_plane, c->d_plane_soa, plane_layout(g.n).stride, s);
  launch_cast_prec32(g.nb, c->d_P, c->d_P32, s);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

sem_status ensure_mixed(sem_ctx* c) {
  if (c->d_st32 != nullptr) return SEM_OK;
  const SemGeom& g = c->g;
  const long long ncls = (long long)g.ux * g.uy * g.uz;
  bool ok = dalloc(&c->d_dcoef_f, ncls * 4) == cudaSuccess &&
            dalloc(&c->d_dinv_f, ncls * (long long)g.n * g.n * g.n) == cudaSuccess &&
            dalloc(&c->d_P32, g.nb) == cudaSuccess && dalloc(&c->d_b32, g.nb) == cudaSuccess &&
            dalloc(&c->d_x32, g.nb) == cudaSuccess && dalloc(&c->d_r32, g.nb) == cudaSuccess &&
            dalloc(&c->d_p32, g.nb) == cudaSuccess && dalloc(&c->d_q32, g.nb) == cudaSuccess &&
            dalloc(&c->d_st32, 1) == cudaSuccess &&
            dalloc(&c->d_coef_f, ncls * coef_offsets(g.n).stride) == cudaSuccess &&
            (!plane_table_used(g.n) || dalloc(&c->d_plane, ncls * plane_layout(g.n).stride) == cudaSuccess) &&
            (g.n != 1 || dalloc(&c->d_coef_soa_f, ncls * coef_offsets(1).stride) == cudaSuccess) &&
            (!elem_supported(g.n) || dalloc(&c->d_plane_soa, ncls * plane_layout(g.n).stride) == cudaSuccess);
  if (!ok) return fail(SEM_ENOMEM, "cannot allocate mixed-precision buffers");
  SEM_CUDA(cudaMemsetAsync(c->d_st32, 0, sizeof(PcgState), c->stream));
  c->tab_f.cls_x = c->tab.cls_x;
  c->tab_f.cls_y = c->tab.cls_y;
  c->tab_f.cls_z = c->tab.cls_z;
  c->tab_f.dcoef = c->d_dcoef_f;
  c->tab_f.dinv = c->d_dinv_f;
  c->tab_f.coef = c->d_coef_f;
  c->tab_f.coef_stride = coef_offsets(g.n).stride;
  c->tab_f.plane = c->d_plane;
  c->tab_f.coef_soa = c->d_coef_soa_f;
  c->tab_f.plane_soa = c->d_plane_soa;
  c->tab_f.ncls = (int)ncls;
  c->tab_f.plane_stride = plane_table_used(g.n) ? plane_layout(g.n).stride : 0;
  sem_status st = cast_tables_f32(c, c->stream);
  if (st != SEM_OK) return st;
  // operator kernel attributes outside any capture
  SEM_CUDA(cudaMemsetAsync(c->d_q32, 0, sizeof(float) * g.nb, c->stream));
  SEM_CUDA(cudaMemsetAsync(c->d_x32, 0, sizeof(float) * g.nb, c->stream));
  launch_tpt_apply<float>(g, c->h1.basis, c->tab_f, c->d_x32, c->d_q32, nullptr, nullptr, c->stream);
  SEM_CUDA(cudaGetLastError());
  SEM_CUDA(prepare_pcg_step<float>(g.nb, &c->step_ok));
  return SEM_OK;
}

sem_status ensure_ctl(sem_ctx* c) {
  if (c->d_ctl != nullptr) return SEM_OK;
  sem_status st = ensure_mixed(c);
  if (st != SEM_OK) return st;
  if (dalloc(&c->d_ctl, 1) != cudaSuccess || dalloc(&c->d_stg, 1) != cudaSuccess)
    return fail(SEM_ENOMEM, "cannot allocate refinement control");
  SEM_CUDA(cudaMemsetAsync(c->d_ctl, 0, sizeof(MixedCtl), c->stream));
  SEM_CUDA(cudaMemsetAsync(c->d_stg, 0, sizeof(PcgState), c->stream));
  SEM_CUDA(cudaStreamSynchronize(c->stream));
  return SEM_OK;
}

sem_status ensure_cubes(sem_ctx* c) {
  if (c->d_c0 != nullptr) return SEM_OK;
  const size_t n3 = (size_t)c->g.nelem * c->g.n * c->g.n * c->g.n;
  if (dalloc(&c->d_c0, n3) != cudaSuccess || dalloc(&c->d_c1, n3) != cudaSuccess ||
      dalloc(&c->d_FtI, n3) != cudaSuccess || dalloc(&c->d_cexp, (size_t)c->g.nelem) != cudaSuccess)
    return fail(SEM_ENOMEM, "cannot allocate element interior scratch");
  return SEM_OK;
}

// fhat~ into out (transformed).  Leaves F~_I in d_FtI for the recovery.
sem_status condense_rhs_t(sem_ctx* c, const double* f, double* out, cudaStream_t s) {
  sem_status st = ensure_cubes(c);
  if (st != SEM_OK) return st;
  const SemGeom& g = c->g;
  const double *mx = c->d_mass, *my = mx + g.Nx, *mz = my + g.Ny;
  launch_load_skeleton(g, mx, my, mz, f, c->d_t1, s);
  launch_skel_transform(g, c->mat(0), c->d_t1, out, s);
  launch_interior_load(g, mx, my, mz, f, c->d_c0, s);
  launch_mode3(g, c->mat(0), c->d_c0, c->d_c1, c->d_cexp, c->d_FtI, nullptr, s);
  launch_condense_faces(g, c->h1.basis, c->tab, c->d_FtI, out, s);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

// Interior recovery from a transformed skeleton solution ut; d_FtI must hold F~_I.
sem_status recover_t(sem_ctx* c, const double* ut, double* u, cudaStream_t s) {
  const SemGeom& g = c->g;
  launch_recover_expand(g, c->h1.basis, c->tab, c->d_FtI, ut, c->d_c0, s);
  launch_mode3(g, c->mat(1), c->d_c0, c->d_c1, c->d_cexp, nullptr, u, s);
  launch_skel_transform(g, c->mat(1), ut, c->d_t2, s);
  launch_unpack(g, c->d_t2, u, 1, s);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

sem_status apply_t(sem_ctx* c, const double* x, double* y, cudaStream_t s) {
  SEM_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * c->g.nb, s));
  launch_tpt_apply<double>(c->g, c->h1.basis, c->tab, x, y, nullptr, nullptr, s,
                           &c->op64);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

// Status message of a solve stopped by a grid-barrier timeout of the one-pass
// CG step (PcgState::bar_fail) rather than by a breakdown of the iteration.
constexpr const char* kBarFailMsg =
    "the one-pass CG step's grid barrier wait ran out (its CTAs were not all resident); "
    "set opts.onepass_step = 0";

// Whether the FP32 CG of a single solve takes the one-pass step.
bool use_step(const sem_ctx* c) { return c->opts.onepass_step != 0 && c->step_ok && !c->step_failed; }

// One FP32 CG iteration on the context's FP32 vectors (st32): operator, then
// update and direction, as one pass with a grid barrier (onepass) or as two
// kernels; e0/e1 (may be null) become event nodes around the operator.
sem_status cg_iter_f32(sem_ctx* c, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, bool onepass) {
  const SemGeom& g = c->g;
  if (e0) cudaEventRecordWithFlags(e0, s, cudaEventRecordExternal);
  launch_tpt_apply<float>(g, c->h1.basis, c->tab_f, c->d_p32, c->d_q32, c->d_partials, c->d_st32, s, &c->op32);
  if (e1) cudaEventRecordWithFlags(e1, s, cudaEventRecordExternal);
  if (onepass) {
    const cudaError_t e = launch_pcg_step<float>(g.nb, c->d_x32, c->d_r32, c->d_p32, c->d_q32, c->d_P32, c->d_partials,
                                                 c->d_st32, s);
    if (e != cudaSuccess) return fail(SEM_ECUDA, std::string("one-pass CG step: ") + cudaGetErrorString(e));
    return SEM_OK;
  }
  launch_pcg_update<float>(g.nb, c->d_r32, c->d_q32, c->d_P32, c->d_partials, c->d_st32, s);
  launch_pcg_dir<float>(g.nb, c->d_x32, c->d_r32, c->d_p32, c->d_q32, c->d_P32, c->d_st32, s);
  return SEM_OK;
}

// One thread: another trip of a device-side CG loop while the solve's flag is
// 0 (running) and fewer than cap trips have run.
__global__ void k_loop_decide(const int* flag, int* trips, int cap, cudaGraphConditionalHandle handle) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int t = ++(*trips);
  cudaGraphSetConditional(handle, (*flag == 0 && t < cap) ? 1u : 0u);
}

// Instantiates *exec from the launches `body` issues on the context stream.
// loop = false: as they are (one replay runs one batch of CG iterations and
// the host decides whether to replay).  loop = true: inside a while node whose
// body ends with k_loop_decide on `flag`, so that one launch runs the whole CG
// on the device; the caller zeroes d_trips before each launch.  *per_trip:
// kernel launches of one pass of the body (counted when it runs).
template <typename F>
sem_status capture_cg(sem_ctx* c, bool loop, const int* flag, int cap, F body, cudaGraphExec_t* exec,
                      long long* per_trip) {
  cudaStream_t s = c->stream;
  cudaGraph_t main_g = nullptr;
  sem_status cst = SEM_OK;
  cudaError_t e = cudaSuccess;
  const long long before = sem_launch_total();
  if (!loop) {
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cst = body(s);
      const cudaError_t e2 = cudaStreamEndCapture(s, &main_g);
      if (e == cudaSuccess) e = e2;
    }
  } else {
    cudaGraphConditionalHandle handle;
    e = cudaGraphCreate(&main_g, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, main_g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t n_loop;
    if (e == cudaSuccess) e = cudaGraphAddNode(&n_loop, main_g, nullptr, nullptr, 0, &cp);
    if (e == cudaSuccess) {
      e = cudaStreamBeginCaptureToGraph(s, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cst = body(s);
        k_loop_decide<<<1, 32, 0, s>>>(flag, c->d_trips, cap, handle);
        sem_count_launch();
        cudaGraph_t tmp = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(s, &tmp);
        if (e == cudaSuccess) e = e2;
      }
    }
  }
  *per_trip = sem_launch_total() - before;
  sem_count_launch(-*per_trip);   // counted at replay instead
  if (e == cudaSuccess && cst == SEM_OK) e = cudaGraphInstantiate(exec, main_g, 0);
  if (main_g) cudaGraphDestroy(main_g);
  if (cst != SEM_OK) return cst;
  if (e != cudaSuccess) return fail(SEM_ECUDA, std::string("CG graph: ") + cudaGetErrorString(e));
  return SEM_OK;
}

// The FP64 CG's graph: check_every iterations; without profiling, inside a
// device-side loop over such batches (one launch per solve).
sem_status build_graph(sem_ctx* c) {
  const int cap = c->opts.maxit / c->opts.check_every + 2;
  if (c->graph != nullptr && c->graph_iters == c->opts.check_every && c->graph_prof == c->prof && c->graph_cap == cap)
    return SEM_OK;
  if (c->prof && (int)c->pev.size() < 2 * c->opts.check_every) {
    while ((int)c->pev.size() < 2 * c->opts.check_every) {
      cudaEvent_t ev;
      SEM_CUDA(cudaEventCreate(&ev));
      c->pev.push_back(ev);
    }
  }
  if (c->graph != nullptr) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  const SemGeom& g = c->g;
  const bool loop = !c->prof;
  const int* flag = reinterpret_cast<const int*>(reinterpret_cast<const char*>(c->d_st) + offsetof(PcgState, done));
  sem_status st = capture_cg(c, loop, flag, cap, [&](cudaStream_t s) -> sem_status {
    for (int it = 0; it < c->opts.check_every; ++it) {
      // external event-record nodes: recorded at every replay, usable for timing
      if (c->prof) cudaEventRecordWithFlags(c->pev[2 * it], s, cudaEventRecordExternal);
      launch_tpt_apply<double>(g, c->h1.basis, c->tab, c->d_p, c->d_q, c->d_partials, c->d_st, s, &c->op64);
      if (c->prof) cudaEventRecordWithFlags(c->pev[2 * it + 1], s, cudaEventRecordExternal);
      launch_pcg_update(g.nb, c->d_r, c->d_q, c->d_P, c->d_partials, c->d_st, s);
      launch_pcg_dir(g.nb, c->d_x, c->d_r, c->d_p, c->d_q, c->d_P, c->d_st, s);
    }
    return SEM_OK;
  }, &c->graph, &c->graph_per_trip);
  if (st != SEM_OK) return st;
  c->graph_iters = c->opts.check_every;
  c->graph_prof = c->prof;
  c->graph_loop = loop;
  c->graph_cap = cap;
  return SEM_OK;
}

// One launch of a device-side CG loop: zero its trip counter, replay, read the
// state record (and the trips, for the launch count).
sem_status run_loop(sem_ctx* c, cudaGraphExec_t exec, long long per_trip, void* host_state, const void* dev_state,
                    size_t state_bytes) {
  cudaStream_t s = c->stream;
  int trips = 0;
  SEM_CUDA(cudaMemsetAsync(c->d_trips, 0, sizeof(int), s));
  SEM_CUDA(cudaGraphLaunch(exec, s));
  SEM_CUDA(cudaMemcpyAsync(host_state, dev_state, state_bytes, cudaMemcpyDeviceToHost, s));
  SEM_CUDA(cudaMemcpyAsync(&trips, c->d_trips, sizeof(int), cudaMemcpyDeviceToHost, s));
  SEM_CUDA(cudaStreamSynchronize(s));
  sem_count_launch((long long)trips * per_trip);
  return SEM_OK;
}

// CG on the transformed condensed system: d_b -> d_x.  warm: d_x holds x0.
sem_status pcg_fp64(sem_ctx* c, bool warm, sem_info* info) {
  const SemGeom& g = c->g;
  cudaStream_t s = c->stream;
  if (warm) {
    sem_status st = apply_t(c, c->d_x, c->d_q, s);
    if (st != SEM_OK) return st;
  }
  launch_pcg_init(g.nb, c->d_b, c->d_r, c->d_p, c->d_q, c->d_x, c->d_P, c->d_partials, c->d_st, c->opts.rtol,
                  c->opts.maxit, warm ? 1 : 0, s);
  SEM_CUDA(cudaGetLastError());
  sem_status st = build_graph(c);
  if (st != SEM_OK) return st;
  if (c->graph_loop) {   // the whole CG in one launch, decided on the device
    st = run_loop(c, c->graph, c->graph_per_trip, c->h_st, c->d_st, sizeof(PcgState));
    if (st != SEM_OK) return st;
  } else {
    SEM_CUDA(cudaMemcpyAsync(c->h_st, c->d_st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
  }
  const int max_batches = c->graph_loop ? 0 : c->opts.maxit / c->opts.check_every + 2;
  for (int b = 0; b < max_batches && c->h_st->done == 0; ++b) {
    const int it0 = c->h_st->iter;
    SEM_CUDA(cudaGraphLaunch(c->graph, s));
    sem_count_launch(c->graph_per_trip);
    SEM_CUDA(cudaMemcpyAsync(c->h_st, c->d_st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    if (c->graph_prof) {
      // operator launches that did work in this batch (later ones exit at once)
      int worked = c->h_st->iter - it0 + (c->h_st->done == 2 ? 1 : 0);
      if (worked > c->graph_iters) worked = c->graph_iters;
      for (int it = 0; it < worked; ++it) {
        float ms = 0.f;
        SEM_CUDA(cudaEventElapsedTime(&ms, c->pev[2 * it], c->pev[2 * it + 1]));
        c->prof_ms += ms;
        c->prof_count += 1;
      }
    }
  }
  launch_pcg_flush<double>(g.nb, c->d_x, c->d_p, c->d_st, s);   // the last x += alpha p
  SEM_CUDA(cudaGetLastError());
  const PcgState& h = *c->h_st;
  if (info) {
    info->iters += h.iter;
    info->rel_res = h.rr0 > 0 ? std::sqrt(h.rr / h.rr0) : 0.0;
  }
  if (h.done == 2) return fail(SEM_EBREAKDOWN, "CG breakdown (p^T A p <= 0 or non-finite values)");
  if (h.done != 1) return fail(SEM_ENOCONV, "CG reached maxit without meeting rtol");
  return SEM_OK;
}

sem_status build_graph32(sem_ctx* c) {
  if (c->graph32 != nullptr && c->graph32_iters == c->opts.check_every && c->graph32_prof == c->prof) return SEM_OK;
  while (c->prof && (int)c->pev32.size() < 2 * c->opts.check_every) {
    cudaEvent_t ev;
    SEM_CUDA(cudaEventCreate(&ev));
    c->pev32.push_back(ev);
  }
  if (c->graph32 != nullptr) {
    cudaGraphExecDestroy(c->graph32);
    c->graph32 = nullptr;
  }
  for (int attempt = 0;; ++attempt) {
    const bool onepass = use_step(c);
    cudaGraph_t graph;
    SEM_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const long long before = sem_launch_total();
    sem_status cst = SEM_OK;
    for (int it = 0; it < c->opts.check_every && cst == SEM_OK; ++it)
      cst = cg_iter_f32(c, c->stream, c->prof ? c->pev32[2 * it] : nullptr, c->prof ? c->pev32[2 * it + 1] : nullptr,
                        onepass);
    c->graph32_launches = sem_launch_total() - before;
    sem_count_launch(-c->graph32_launches);
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (e == cudaSuccess && cst == SEM_OK) {
      e = cudaGraphInstantiate(&c->graph32, graph, 0);
      cudaGraphDestroy(graph);
      if (e == cudaSuccess) break;
    } else if (e == cudaSuccess) {
      cudaGraphDestroy(graph);
    }
    if (onepass && attempt == 0) {   // a graph with the one-pass step could not be built: two passes
      cudaGetLastError();
      c->step_failed = true;
      continue;
    }
    if (cst != SEM_OK) return cst;
    return fail(SEM_ECUDA, std::string("FP32 CG graph: ") + cudaGetErrorString(e));
  }
  c->graph32_iters = c->opts.check_every;
  c->graph32_prof = c->prof;
  return SEM_OK;
}

// Iterative refinement: x_{k+1} = x_k + ||r_k|| c_k, where c_k solves
// A c = r_k / ||r_k|| by FP32 CG to a relative residual inner_rtol, and
// r_{k+1} = b - A x_{k+1} is formed with the FP64 operator.  d_b -> d_x.
sem_status pcg_mixed(sem_ctx* c, bool warm, sem_info* info) {
  const SemGeom& g = c->g;
  cudaStream_t s = c->stream;
  sem_status st = ensure_mixed(c);
  if (st != SEM_OK) return st;
  st = build_graph32(c);
  if (st != SEM_OK) return st;
  c->refine_hist.clear();
  if (warm) {
    st = apply_t(c, c->d_x, c->d_q, s);
  } else {
    SEM_CUDA(cudaMemsetAsync(c->d_x, 0, sizeof(double) * g.nb, s));
    SEM_CUDA(cudaMemsetAsync(c->d_q, 0, sizeof(double) * g.nb, s));
  }
  if (st != SEM_OK) return st;
  // ||b|| as the reference of the stopping rule
  SEM_CUDA(cudaMemsetAsync(c->d_t2, 0, sizeof(double) * g.nb, s));
  launch_ir_residual(g.nb, c->d_b, c->d_t2, c->d_r, c->d_partials, c->d_st, s);
  SEM_CUDA(cudaMemcpyAsync(c->h_st, c->d_st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  SEM_CUDA(cudaStreamSynchronize(s));
  const double bb = c->h_st->rr;
  launch_ir_residual(g.nb, c->d_b, c->d_q, c->d_r, c->d_partials, c->d_st, s);
  int total = 0, refinements = 0;
  double rel = 1.0, prev = 1e300;
  sem_status result = SEM_ENOCONV;
  for (;;) {
    SEM_CUDA(cudaMemcpyAsync(c->h_st, c->d_st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    const double rr = c->h_st->rr;
    if (!std::isfinite(rr)) { result = SEM_EBREAKDOWN; break; }
    rel = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
    c->refine_hist.push_back(rel);
    if (rel <= c->opts.rtol) { result = SEM_OK; break; }
    if (refinements >= c->opts.max_refine || total >= c->opts.maxit) break;
    if (!(rel < 0.9 * prev)) break;   // refinement stagnated at the FP32 accuracy limit
    prev = rel;
    const double norm = std::sqrt(rr);
    launch_scale_to_f32(g.nb, c->d_r, 1.0 / norm, c->d_b32, s);
    launch_pcg_init<float>(g.nb, c->d_b32, c->d_r32, c->d_p32, c->d_q32, c->d_x32, c->d_P32, c->d_partials,
                           c->d_st32, c->opts.inner_rtol, c->opts.maxit - total, 0, s);
    SEM_CUDA(cudaMemcpyAsync(c->h_st, c->d_st32, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; b < c->opts.maxit / c->opts.check_every + 2 && c->h_st->done == 0; ++b) {
      const int it0 = c->h_st->iter;
      SEM_CUDA(cudaGraphLaunch(c->graph32, s));
      sem_count_launch(c->graph32_launches);
      SEM_CUDA(cudaMemcpyAsync(c->h_st, c->d_st32, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
      SEM_CUDA(cudaStreamSynchronize(s));
      if (c->graph32_prof) {
        int worked = c->h_st->iter - it0 + (c->h_st->done == 2 ? 1 : 0);
        if (worked > c->graph32_iters) worked = c->graph32_iters;
        for (int it = 0; it < worked; ++it) {
          float ms = 0.f;
          SEM_CUDA(cudaEventElapsedTime(&ms, c->pev32[2 * it], c->pev32[2 * it + 1]));
          c->prof_ms += ms;
          c->prof_count += 1;
        }
      }
    }
    const int inner = c->h_st->iter;
    total += inner;
    ++refinements;
    if (c->h_st->done == 2 && inner == 0) { result = SEM_EBREAKDOWN; break; }
    launch_pcg_flush<float>(g.nb, c->d_x32, c->d_p32, c->d_st32, s);
    launch_ir_update(g.nb, c->d_x, c->d_x32, norm, s);
    st = apply_t(c, c->d_x, c->d_q, s);
    if (st != SEM_OK) return st;
    launch_ir_residual(g.nb, c->d_b, c->d_q, c->d_r, c->d_partials, c->d_st, s);
    SEM_CUDA(cudaGetLastError());
  }
  if (info) {
    info->iters += total;
    info->refinements = refinements;
    info->rel_res = rel;
  }
  if (result == SEM_EBREAKDOWN)
    return fail(result, c->h_st->bar_fail ? kBarFailMsg : "CG breakdown or non-finite residual in the refinement");
  if (result != SEM_OK) return fail(result, "refinement did not reach rtol (maxit, max_refine or stagnation)");
  return SEM_OK;
}

// Mixed precision with reliable updates: one FP32 CG whose search direction
// is kept across refinement steps.  A refinement step (when the FP32
// recursive residual has fallen by reliable_delta since the previous step, or
// the FP32 CG stops) adds the FP32 correction to the FP64 iterate, recomputes the
// true residual b - A x with the FP64 operator and restarts the FP32
// recursion from it (rho, |r|^2) without resetting the direction.
// One loop trip of the reliable-update mixed solve: the refinement step
// (when due; every kernel gated on the device) and check_every FP32 CG
// iterations, with event nodes around the FP32 operator when profiling.
sem_status build_graph32m(sem_ctx* c) {
  const int cap = c->opts.maxit / c->opts.check_every + 2 + c->opts.max_refine;
  if (c->graph32m != nullptr && c->graph32m_iters == c->opts.check_every && c->graph32m_prof == c->prof &&
      c->graph32m_cap == cap)
    return SEM_OK;
  while (c->prof && (int)c->pev32.size() < 2 * c->opts.check_every) {
    cudaEvent_t ev;
    SEM_CUDA(cudaEventCreate(&ev));
    c->pev32.push_back(ev);
  }
  if (c->graph32m != nullptr) {
    cudaGraphExecDestroy(c->graph32m);
    c->graph32m = nullptr;
  }
  const SemGeom& g = c->g;
  const bool loop = !c->prof;
  const int* flag = reinterpret_cast<const int*>(reinterpret_cast<const char*>(c->d_ctl) + offsetof(MixedCtl, finished));
  sem_status st = SEM_OK;
  for (int attempt = 0;; ++attempt) {
    const bool onepass = use_step(c);
    st = capture_cg(c, loop, flag, cap, [&](cudaStream_t s) -> sem_status {
      launch_mixed_step(g, c->h1.basis, c->tab, &c->op64, c->d_b, c->d_x, c->d_q, c->d_r, c->d_x32, c->d_r32,
                        c->d_p32, c->d_q32, c->d_P32, c->d_partials, c->d_ctl, c->d_st32, c->d_stg, s);
      sem_status cst = SEM_OK;
      for (int it = 0; it < c->opts.check_every && cst == SEM_OK; ++it)
        cst = cg_iter_f32(c, s, c->prof ? c->pev32[2 * it] : nullptr, c->prof ? c->pev32[2 * it + 1] : nullptr,
                          onepass);
      return cst;
    }, &c->graph32m, &c->graph32m_per_trip);
    if (st == SEM_OK || !onepass || attempt > 0) break;
    cudaGetLastError();   // a graph with the one-pass step could not be built: two passes
    c->step_failed = true;
  }
  if (st != SEM_OK) return st;
  c->graph32m_launches = c->graph32m_per_trip;
  c->graph32m_iters = c->opts.check_every;
  c->graph32m_prof = c->prof;
  c->graph32m_loop = loop;
  c->graph32m_cap = cap;
  return SEM_OK;
}

// The first part of a reliable-update mixed solve, d_b -> d_x: ||b||^2 into
// d_st, r_0 = b - A x_0 (x_0 = d_x when warm, else 0), the FP32 CG on r_0 and
// the refinement control.  Shared by single and batched solves.
sem_status mixed_prologue(sem_ctx* c, bool warm, cudaStream_t s) {
  const long long nb = c->g.nb;
  SEM_CUDA(cudaMemsetAsync(c->d_q, 0, sizeof(double) * nb, s));
  launch_ir_residual(nb, c->d_b, c->d_q, c->d_r, c->d_partials, c->d_st, s);   // ||b||^2
  if (warm) {
    sem_status st = apply_t(c, c->d_x, c->d_q, s);
    if (st != SEM_OK) return st;
    launch_ir_residual(nb, c->d_b, c->d_q, c->d_r, c->d_partials, c->d_stg, s);
  } else {
    SEM_CUDA(cudaMemsetAsync(c->d_x, 0, sizeof(double) * nb, s));
  }
  launch_scale_to_f32(nb, c->d_r, 1.0, c->d_b32, s);
  launch_pcg_init<float>(nb, c->d_b32, c->d_r32, c->d_p32, c->d_q32, c->d_x32, c->d_P32, c->d_partials, c->d_st32,
                         c->opts.rtol, c->opts.maxit, 0, s);
  // reliable_delta 0: the measured best on GB300, 0.03 at p = 2 (where the FP32 CG loses the most iterations
  // to FP32 rounding and a refinement step costs four FP32 iterations), 0.01 otherwise
  const double delta = c->opts.reliable_delta > 0.0 ? c->opts.reliable_delta : (c->g.n == 1 ? 0.03 : 0.01);
  launch_mixed_start(c->d_ctl, c->d_st, c->d_st32, c->opts.rtol, delta, c->opts.max_refine, s);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

// Reliable updates: one FP32 CG kept across the FP64 refinement steps; the
// step is triggered on the device when the FP32 residual has fallen by
// reliable_delta and replaces the FP32 residual by the true one (residual
// replacement, direction kept), all decided by the kernels of
// launch_mixed_step; the host replays one loop trip per graph launch and
// reads the control record.  d_b -> d_x.
sem_status pcg_mixed_reliable(sem_ctx* c, bool warm, sem_info* info) {
  const SemGeom& g = c->g;
  cudaStream_t s = c->stream;
  sem_status st = ensure_ctl(c);
  if (st != SEM_OK) return st;
  st = build_graph32m(c);
  if (st != SEM_OK) return st;
  st = mixed_prologue(c, warm, s);
  if (st != SEM_OK) return st;
  MixedCtl* hc = &c->h_ctl;
  if (c->graph32m_loop) {   // the whole refinement-and-CG loop in one launch, decided on the device
    st = run_loop(c, c->graph32m, c->graph32m_per_trip, hc, c->d_ctl, sizeof(MixedCtl));
    if (st != SEM_OK) return st;
  }
  const int cap = c->graph32m_loop ? 0 : c->opts.maxit / c->opts.check_every + 2 + c->opts.max_refine;
  int it0 = 0;
  for (int trip = 0; trip < cap; ++trip) {
    SEM_CUDA(cudaMemcpyAsync(hc, c->d_ctl, sizeof(MixedCtl), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    if (hc->finished != 0) break;
    SEM_CUDA(cudaGraphLaunch(c->graph32m, s));
    sem_count_launch(c->graph32m_launches);
    SEM_CUDA(cudaMemcpyAsync(c->h_st, c->d_st32, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    if (c->graph32m_prof) {
      int worked = c->h_st->iter - it0 + (c->h_st->done == 2 ? 1 : 0);
      if (worked > c->graph32m_iters) worked = c->graph32m_iters;
      if (worked < 0) worked = 0;
      for (int it = 0; it < worked; ++it) {
        float ms = 0.f;
        SEM_CUDA(cudaEventElapsedTime(&ms, c->pev32[2 * it], c->pev32[2 * it + 1]));
        c->prof_ms += ms;
        c->prof_count += 1;
      }
    }
    it0 = c->h_st->iter;
  }
  // a correction not yet folded in (the loop stopped between refinement steps)
  launch_pcg_flush<float>(g.nb, c->d_x32, c->d_p32, c->d_st32, s);
  launch_ir_update(g.nb, c->d_x, c->d_x32, 1.0, s);
  SEM_CUDA(cudaMemsetAsync(c->d_x32, 0, sizeof(float) * g.nb, s));
  SEM_CUDA(cudaMemcpyAsync(hc, c->d_ctl, sizeof(MixedCtl), cudaMemcpyDeviceToHost, s));
  SEM_CUDA(cudaMemcpyAsync(c->h_st, c->d_st32, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  SEM_CUDA(cudaStreamSynchronize(s));
  const int last = std::min(hc->refinements, kMixedHist - 1);
  c->refine_hist.assign(hc->hist, hc->hist + last + 1);
  if (info) {
    info->iters += c->h_st->iter;
    info->refinements = hc->refinements;
    info->rel_res = hc->hist[last];
  }
  if (hc->finished == 2)
    return fail(SEM_EBREAKDOWN, c->h_st->bar_fail ? kBarFailMsg : "CG breakdown or non-finite residual in the refinement");
  if (hc->finished != 1) return fail(SEM_ENOCONV, "refinement did not reach rtol (maxit, max_refine or stagnation)");
  return SEM_OK;
}

void free_ctx(sem_ctx* c) {
  if (c == nullptr) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->graph32) cudaGraphExecDestroy(c->graph32);
  if (c->graph32m) cudaGraphExecDestroy(c->graph32m);
  void* ptrs32[] = {c->d_dcoef_f, c->d_dinv_f, c->d_P32, c->d_b32, c->d_x32, c->d_r32, c->d_p32, c->d_q32, c->d_st32,
                    c->d_coef_f, c->d_coef, c->d_plane, c->d_ctl, c->d_stg, c->d_coef_soa, c->d_coef_soa_f,
                    c->d_plane_soa, c->d_hf, c->d_hu};
  for (void* p : ptrs32)
    if (p) cudaFree(p);
  for (cudaEvent_t ev : c->pev32) cudaEventDestroy(ev);
  void* ptrs_cmp[] = {c->d_cmpK, c->d_cmp, c->d_cst, c->d_cdiag, c->d_Pdc, c->d_mmc, c->d_cls_elems, c->d_mmcU,
                      c->d_mmcY};
  for (void* p : ptrs_cmp)
    if (p) cudaFree(p);
  if (c->cublas) cublasDestroy(c->cublas);
  void* ptrs_adj[] = {c->d_h, c->d_K, c->d_full, c->d_E, c->d_grad};
  for (void* p : ptrs_adj)
    if (p) cudaFree(p);
  if (c->d_trips) cudaFree(c->d_trips);
  if (c->d_ev) cudaFree(c->d_ev);
  void* ptrs[] = {c->d_cls, c->d_uw, c->d_dcoef, c->d_dinv, c->d_mats, c->d_mass, c->d_P, c->d_x, c->d_r,
                  c->d_p, c->d_q, c->d_b, c->d_t1, c->d_t2, c->d_c0, c->d_c1, c->d_FtI, c->d_cexp, c->d_partials, c->d_st};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_st) cudaFreeHost(c->h_st);
  for (cudaEvent_t ev : c->pev) cudaEventDestroy(ev);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->stream) cudaStreamDestroy(c->stream);
  cudaSetDevice(prev);
  delete c;
}

// A context and the current device: kernels launch on the current device and
// read the context's tables and the caller's vectors on c->device, so an entry
// point that launches refuses to run while another device is current.
sem_status check_ctx(const sem_ctx* c) {
  if (c == nullptr) return fail(SEM_EINVAL, "null context");
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return fail(SEM_EINVAL, "cannot query the current device");
  }
  if (cur != c->device)
    return fail(SEM_EINVAL, "the current device (" + std::to_string(cur) + ") is not the context's device (" +
                                std::to_string(c->device) + ")");
  return SEM_OK;
}

// A caller vector of `elem`-byte entries: not null, aligned to its entry size,
// and device memory of the context's device (or managed memory), so that no
// kernel is launched on a host pointer or on another GPU's memory.
sem_status check_vec(const sem_ctx* c, const void* p, size_t elem, const char* name) {
  if (p == nullptr) return fail(SEM_EINVAL, std::string(name) + " is null");
  if (reinterpret_cast<uintptr_t>(p) % elem != 0)
    return fail(SEM_EINVAL, std::string(name) + " is not aligned to its entry size");
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();   // the query's error is not sticky: clear it
    return fail(SEM_EINVAL, std::string(name) + " is not a CUDA address");
  }
  if (a.type == cudaMemoryTypeManaged) return SEM_OK;
  if (a.type != cudaMemoryTypeDevice) return fail(SEM_EINVAL, std::string(name) + " is not device memory");
  if (a.device != c->device) return fail(SEM_EINVAL, std::string(name) + " is on another device than the context");
  return SEM_OK;
}

// check_vec of vector p (entries of type T) in an entry point whose context is `c`
#define SEM_CHECK_VEC(p, T)                                        \
  do {                                                             \
    const sem_status st_ = check_vec(c, (p), sizeof(T), #p);        \
    if (st_ != SEM_OK) return st_;                                 \
  } while (0)

// NVTX range over one entry point or phase of it: named in profiler timelines
// and usable as a profiler filter; without a tool attached it costs a check.
struct NvtxScope {
  explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
  NvtxScope(const NvtxScope&) = delete;
  NvtxScope& operator=(const NvtxScope&) = delete;
};

}  // namespace

extern "C" {

void sem_default_opts(sem_opts* o) {
  if (o == nullptr) return;
  o->rtol = 1e-10;
  o->maxit = 50000;
  o->precision = SEM_PREC_FP64;
  o->check_every = 16;
  o->inner_rtol = 1e-4;
  o->max_refine = 40;
  o->mixed_scheme = 1;
  o->reliable_delta = 0.0;   // automatic (by degree)
  o->deterministic = 1;
  o->onepass_step = 1;
}

static sem_status check_opts(const sem_opts* o) {
  if (!(o->rtol > 0.0 && o->rtol < 1.0)) return fail(SEM_EINVAL, "rtol must be in (0, 1)");
  if (o->maxit < 1) return fail(SEM_EINVAL, "maxit must be >= 1");
  if (o->check_every < 1 || o->check_every > 1024) return fail(SEM_EINVAL, "check_every must be in [1, 1024]");
  if (o->precision != SEM_PREC_FP64 && o->precision != SEM_PREC_MIXED) return fail(SEM_EINVAL, "unknown precision");
  if (!(o->inner_rtol > 0.0 && o->inner_rtol < 1.0)) return fail(SEM_EINVAL, "inner_rtol must be in (0, 1)");
  if (o->max_refine < 1) return fail(SEM_EINVAL, "max_refine must be >= 1");
  if (o->mixed_scheme != 0 && o->mixed_scheme != 1) return fail(SEM_EINVAL, "mixed_scheme must be 0 or 1");
  if (!(o->reliable_delta == 0.0 || (o->reliable_delta > 0.0 && o->reliable_delta < 1.0)))
    return fail(SEM_EINVAL, "reliable_delta must be 0 (automatic) or in (0, 1)");
  if (o->deterministic != 0 && o->deterministic != 1) return fail(SEM_EINVAL, "deterministic must be 0 or 1");
  if (o->onepass_step != 0 && o->onepass_step != 1) return fail(SEM_EINVAL, "onepass_step must be 0 or 1");
  return SEM_OK;
}

namespace {
void drop_graph(sem_ctx* c, bool mixed);
}

// With opts.deterministic the FP64 operator sums the edge and vertex outputs
// in a fixed order through per-element scratch (allocated here on first use)
// instead of atomics; its configuration carries the scratch pointer.
static sem_status sync_deterministic(sem_ctx* c) {
  if (c->opts.deterministic && c->d_ev == nullptr) {
    const size_t count = (size_t)c->g.nelem * (12 * (size_t)c->g.n + 8);
    if (cudaMalloc((void**)&c->d_ev, count * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      c->d_ev = nullptr;
      return fail(SEM_ENOMEM, "cannot allocate the fixed-order edge/vertex scratch");
    }
  }
  c->op64.ev = c->opts.deterministic ? c->d_ev : nullptr;
  return SEM_OK;
}

sem_status sem_setup(sem_ctx** out, int p, int mx, int my, int mz, const double* hx, const double* hy,
                     const double* hz, double lambda, const sem_opts* opts) {
  t_err.clear();
  NvtxScope nvtx_("sem_setup");
  if (out == nullptr) return fail(SEM_EINVAL, "out is null");
  *out = nullptr;
  if (p < 2 || p > 32) return fail(SEM_EINVAL, "p must be in [2, 32]");
  if (mx < 1 || my < 1 || mz < 1) return fail(SEM_EINVAL, "element counts must be >= 1");
  if (!valid_widths(hx, mx) || !valid_widths(hy, my) || !valid_widths(hz, mz))
    return fail(SEM_EINVAL, "element widths must be positive and finite");
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return fail(SEM_EINVAL, "lambda must be finite and >= 0");
  sem_opts o;
  sem_default_opts(&o);
  if (opts) o = *opts;
  sem_status vs = check_opts(&o);
  if (vs != SEM_OK) return vs;

  sem_ctx* c = new sem_ctx();
  cudaGetDevice(&c->device);
  c->opts = o;
  c->lambda = lambda;
  std::string err;
  if (!sem_build_1d(p, &c->h1, &err)) {
    delete c;
    return fail(SEM_EINVAL, err);
  }
  c->hx.assign(hx, hx + mx);
  c->hy.assign(hy, hy + my);
  c->hz.assign(hz, hz + mz);
  build_classes(c->hx, &c->uxw, &c->clsx);
  build_classes(c->hy, &c->uyw, &c->clsy);
  build_classes(c->hz, &c->uzw, &c->clsz);
  SemGeom& g = c->g;
  const int n = p - 1;
  g.p = p;
  g.n = n;
  g.mx = mx;
  g.my = my;
  g.mz = mz;
  g.ux = (int)c->uxw.size();
  g.uy = (int)c->uyw.size();
  g.uz = (int)c->uzw.size();
  g.nelem = (long long)mx * my * mz;
  g.slow = (g.ux >= g.uy && g.ux >= g.uz && g.ux > 1) ? 0 : ((g.uy >= g.uz && g.uy > 1) ? 1 : 2);
  const long long n2 = (long long)n * n;
  const long long cnt[7] = {(long long)(mx + 1) * my * mz * n2,       (long long)mx * (my + 1) * mz * n2,
                            (long long)mx * my * (mz + 1) * n2,       (long long)mx * (my + 1) * (mz + 1) * n,
                            (long long)(mx + 1) * my * (mz + 1) * n,  (long long)(mx + 1) * (my + 1) * mz * n,
                            (long long)(mx + 1) * (my + 1) * (mz + 1)};
  g.off[0] = 0;
  for (int b = 0; b < 7; ++b) g.off[b + 1] = g.off[b] + cnt[b];
  g.nb = g.off[7];
#ifdef SEM_DEBUG
  g.dbg_bound = g.nb;
#endif
  if (g.nb >= (1LL << 31)) {
    delete c;
    return fail(SEM_ENOTSUP, "skeleton too large: N_B must be below 2^31");
  }
  g.Nx = (long long)mx * p + 1;
  g.Ny = (long long)my * p + 1;
  g.Nz = (long long)mz * p + 1;

  std::vector<double> mass, mxv, myv, mzv;
  axis_mass_coords(p, c->hx, c->h1.x, c->h1.w, &mxv, &c->xc);
  axis_mass_coords(p, c->hy, c->h1.x, c->h1.w, &myv, &c->yc);
  axis_mass_coords(p, c->hz, c->h1.x, c->h1.w, &mzv, &c->zc);
  mass.insert(mass.end(), mxv.begin(), mxv.end());
  mass.insert(mass.end(), myv.begin(), myv.end());
  mass.insert(mass.end(), mzv.begin(), mzv.end());

  // transform matrices, row-major n x n
  std::vector<double> mats(4 * n2);
  const std::vector<double>& V = c->h1.V;
  for (int r = 0; r < n; ++r)
    for (int q = 0; q < n; ++q) {
      mats[0 * n2 + r * n + q] = V[q * n + r];                      // S_II = V^T
      mats[1 * n2 + r * n + q] = V[r * n + q];                      // V
      mats[2 * n2 + r * n + q] = V[q * n + r] * c->h1.w[q + 1];     // S_II^-T = V^T M_II
      mats[3 * n2 + r * n + q] = c->h1.w[r + 1] * V[r * n + q];     // S_II^-1 = M_II V
    }

  const long long ncls = (long long)g.ux * g.uy * g.uz;
  std::vector<int> cls;
  cls.insert(cls.end(), c->clsx.begin(), c->clsx.end());
  cls.insert(cls.end(), c->clsy.begin(), c->clsy.end());
  cls.insert(cls.end(), c->clsz.begin(), c->clsz.end());
  std::vector<double> uw;
  uw.insert(uw.end(), c->uxw.begin(), c->uxw.end());
  uw.insert(uw.end(), c->uyw.begin(), c->uyw.end());
  uw.insert(uw.end(), c->uzw.begin(), c->uzw.end());

  bool ok = dalloc(&c->d_cls, cls.size()) == cudaSuccess && dalloc(&c->d_uw, uw.size()) == cudaSuccess &&
            dalloc(&c->d_dcoef, ncls * 4) == cudaSuccess && dalloc(&c->d_dinv, ncls * n2 * n) == cudaSuccess &&
            dalloc(&c->d_coef, ncls * coef_offsets(n).stride) == cudaSuccess &&
            (n != 1 || dalloc(&c->d_coef_soa, ncls * coef_offsets(1).stride) == cudaSuccess) &&
            dalloc(&c->d_mats, mats.size()) == cudaSuccess && dalloc(&c->d_mass, mass.size()) == cudaSuccess &&
            dalloc(&c->d_P, g.nb) == cudaSuccess && dalloc(&c->d_x, g.nb) == cudaSuccess &&
            dalloc(&c->d_r, g.nb) == cudaSuccess && dalloc(&c->d_p, g.nb) == cudaSuccess &&
            dalloc(&c->d_q, g.nb) == cudaSuccess && dalloc(&c->d_b, g.nb) == cudaSuccess &&
            dalloc(&c->d_t1, g.nb) == cudaSuccess && dalloc(&c->d_t2, g.nb) == cudaSuccess &&
            dalloc(&c->d_partials, kPartials) == cudaSuccess && dalloc(&c->d_st, 1) == cudaSuccess &&
            dalloc(&c->d_trips, 1) == cudaSuccess &&
            cudaMallocHost((void**)&c->h_st, sizeof(PcgState)) == cudaSuccess;
  if (!ok) {
    free_ctx(c);
    return fail(SEM_ENOMEM, "device allocation failed in sem_setup");
  }
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
  cudaStream_t s = c->stream;
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_cls, cls.data(), cls.size() * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_uw, uw.data(), uw.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_mats, mats.data(), mats.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_mass, mass.data(), mass.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_st, 0, sizeof(PcgState), s);
  if (e != cudaSuccess) {
    free_ctx(c);
    return fail(SEM_ECUDA, std::string("sem_setup: ") + cudaGetErrorString(e));
  }
  c->tab.cls_x = c->d_cls;
  c->tab.cls_y = c->d_cls + mx;
  c->tab.cls_z = c->d_cls + mx + my;
  c->tab.dcoef = c->d_dcoef;
  c->tab.dinv = c->d_dinv;
  c->tab.coef = c->d_coef;
  c->tab.coef_stride = coef_offsets(n).stride;
  c->tab.coef_soa = c->d_coef_soa;
  c->tab.ncls = (int)ncls;
  sem_status st = compute_tables(c, s);
  if (st == SEM_OK) st = sync_deterministic(c);
  if (st == SEM_OK) {
    // warm the operator kernel's attributes outside any graph capture
    st = apply_t(c, c->d_P, c->d_t2, s);
  }
  if (st == SEM_OK) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = fail(SEM_ECUDA, std::string("sem_setup: ") + cudaGetErrorString(e));
  }
  if (st != SEM_OK) {
    std::string keep = t_err;
    free_ctx(c);
    t_err = keep;
    return st;
  }
  *out = c;
  return SEM_OK;
}

sem_status sem_set_lambda(sem_ctx* c, double lambda) {
  t_err.clear();
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return fail(SEM_EINVAL, "lambda must be finite and >= 0");
  c->lambda = lambda;
  sem_status st = compute_tables(c, c->stream);
  if (st != SEM_OK) return st;
  SEM_CUDA(cudaStreamSynchronize(c->stream));
  return SEM_OK;
}

sem_status sem_set_opts(sem_ctx* c, const sem_opts* opts) {
  t_err.clear();
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  sem_opts o;
  sem_default_opts(&o);
  if (opts) o = *opts;
  sem_status vs = check_opts(&o);
  if (vs != SEM_OK) return vs;
  const bool det_changed = (o.deterministic != 0) != (c->opts.deterministic != 0) ||
                           (o.onepass_step != 0) != (c->opts.onepass_step != 0);
  c->opts = o;
  if (det_changed) {   // the captured operator or CG-step launches change
    drop_graph(c, false);
    drop_graph(c, true);
  }
  return sync_deterministic(c);
}

sem_status sem_skeleton_size(const sem_ctx* c, long long* nb) {
  if (c == nullptr || nb == nullptr) return fail(SEM_EINVAL, "null argument");
  *nb = c->g.nb;
  return SEM_OK;
}

sem_status sem_grid_size(const sem_ctx* c, long long* n) {
  if (c == nullptr || n == nullptr) return fail(SEM_EINVAL, "null argument");
  *n = c->g.Nx * c->g.Ny * c->g.Nz;
  return SEM_OK;
}

sem_status sem_node_coords(const sem_ctx* c, double* x, double* y, double* z) {
  if (c == nullptr || x == nullptr || y == nullptr || z == nullptr) return fail(SEM_EINVAL, "null argument");
  std::memcpy(x, c->xc.data(), c->xc.size() * sizeof(double));
  std::memcpy(y, c->yc.data(), c->yc.size() * sizeof(double));
  std::memcpy(z, c->zc.data(), c->zc.size() * sizeof(double));
  return SEM_OK;
}

sem_status sem_get_basis(const sem_ctx* c, double* gx, double* gw, double* lam, double* V) {
  if (c == nullptr) return fail(SEM_EINVAL, "null context");
  const SemHost1D& h = c->h1;
  if (gx) std::memcpy(gx, h.x.data(), h.x.size() * sizeof(double));
  if (gw) std::memcpy(gw, h.w.data(), h.w.size() * sizeof(double));
  if (lam) std::memcpy(lam, h.lam.data(), h.lam.size() * sizeof(double));
  if (V) std::memcpy(V, h.V.data(), h.V.size() * sizeof(double));
  return SEM_OK;
}

sem_status sem_apply_condensed(sem_ctx* c, const double* uB, double* vB, sem_space space, void* stream) {
  t_err.clear();
  NvtxScope nvtx_("sem_apply_condensed");
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  SEM_CHECK_VEC(uB, double);
  SEM_CHECK_VEC(vB, double);
  if (uB == vB) return fail(SEM_EINVAL, "uB and vB must not alias");
  cudaStream_t s = (cudaStream_t)stream;
  if (space == SEM_SPACE_TRANSFORMED) return apply_t(c, uB, vB, s);
  if (space != SEM_SPACE_NODAL) return fail(SEM_EINVAL, "unknown space");
  launch_skel_transform(c->g, c->mat(2), uB, c->d_t1, s);
  sem_status st = apply_t(c, c->d_t1, c->d_t2, s);
  if (st != SEM_OK) return st;
  launch_skel_transform(c->g, c->mat(3), c->d_t2, vB, s);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

sem_status sem_apply_condensed_f32(sem_ctx* c, const float* uB, float* vB, void* stream) {
  t_err.clear();
  NvtxScope nvtx_("sem_apply_condensed_f32");
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  SEM_CHECK_VEC(uB, float);
  SEM_CHECK_VEC(vB, float);
  if ((const void*)uB == (const void*)vB) return fail(SEM_EINVAL, "uB and vB must not alias");
  sem_status st = ensure_mixed(c);
  if (st != SEM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  SEM_CUDA(cudaStreamSynchronize(c->stream));   // FP32 tables are prepared on the context stream
  SEM_CUDA(cudaMemsetAsync(vB, 0, sizeof(float) * c->g.nb, s));
  launch_tpt_apply<float>(c->g, c->h1.basis, c->tab_f, uB, vB, nullptr, nullptr, s,
                          &c->op32);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

sem_status sem_condense_rhs(sem_ctx* c, const double* f, double* fB, sem_space space, void* stream) {
  t_err.clear();
  NvtxScope nvtx_("sem_condense_rhs");
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  SEM_CHECK_VEC(f, double);
  SEM_CHECK_VEC(fB, double);
  if (space != SEM_SPACE_NODAL && space != SEM_SPACE_TRANSFORMED) return fail(SEM_EINVAL, "unknown space");
  cudaStream_t s = (cudaStream_t)stream;
  sem_status st = condense_rhs_t(c, f, fB, s);
  if (st != SEM_OK) return st;
  if (space == SEM_SPACE_NODAL) {
    launch_skel_transform(c->g, c->mat(3), fB, fB, s);
    SEM_CUDA(cudaGetLastError());
  }
  return SEM_OK;
}

sem_status sem_precond_diag(sem_ctx* c, double* diag, void* stream) {
  t_err.clear();
  NvtxScope nvtx_("sem_precond_diag");
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  SEM_CHECK_VEC(diag, double);
  cudaStream_t s = (cudaStream_t)stream;
  SEM_CUDA(cudaMemsetAsync(diag, 0, sizeof(double) * c->g.nb, s));
  launch_precond_diag(c->g, c->h1.basis, c->tab, diag, s);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

sem_status sem_recover_interior(sem_ctx* c, const double* f, const double* uB, sem_space space, double* u,
                                void* stream) {
  t_err.clear();
  NvtxScope nvtx_("sem_recover_interior");
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  SEM_CHECK_VEC(f, double);
  SEM_CHECK_VEC(uB, double);
  SEM_CHECK_VEC(u, double);
  if (space != SEM_SPACE_NODAL && space != SEM_SPACE_TRANSFORMED) return fail(SEM_EINVAL, "unknown space");
  cudaStream_t s = (cudaStream_t)stream;
  // F~_I for this f (the condensed load itself is discarded)
  sem_status st = condense_rhs_t(c, f, c->d_b, s);
  if (st != SEM_OK) return st;
  const double* ut = uB;
  if (space == SEM_SPACE_NODAL) {
    launch_skel_transform(c->g, c->mat(2), uB, c->d_x, s);
    ut = c->d_x;
  }
  return recover_t(c, ut, u, s);
}

sem_status sem_solve(sem_ctx* c, const double* f, double* u, const double* u0, sem_info* info, void* stream) {
  t_err.clear();
  NvtxScope nvtx_("sem_solve");
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  SEM_CHECK_VEC(f, double);
  SEM_CHECK_VEC(u, double);
  if (u0 != nullptr) SEM_CHECK_VEC(u0, double);
  const auto t0 = std::chrono::steady_clock::now();
  if (info) std::memset(info, 0, sizeof(*info));
  cudaStream_t us = (cudaStream_t)stream;
  SEM_CUDA(cudaEventRecord(c->ev_in, us));
  SEM_CUDA(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
  cudaStream_t s = c->stream;
  sem_status st;
  {
    NvtxScope phase("condense");
    st = condense_rhs_t(c, f, c->d_b, s);
  }
  if (st != SEM_OK) return st;
  if (u0) launch_skel_transform(c->g, c->mat(2), u0, c->d_x, s);
  sem_status cg;
  {
    NvtxScope phase(c->opts.precision == SEM_PREC_MIXED ? "pcg_mixed" : "pcg_fp64");
    if (c->opts.precision == SEM_PREC_MIXED)
      cg = c->opts.mixed_scheme == 1 ? pcg_mixed_reliable(c, u0 != nullptr, info) : pcg_mixed(c, u0 != nullptr, info);
    else
      cg = pcg_fp64(c, u0 != nullptr, info);
  }
  if (cg != SEM_OK && cg != SEM_ENOCONV && cg != SEM_EBREAKDOWN) return cg;
  std::string cg_err = t_err;
  {
    NvtxScope phase("recover");
    st = recover_t(c, c->d_x, u, s);
  }
  if (st != SEM_OK) return st;
  SEM_CUDA(cudaEventRecord(c->ev_out, s));
  SEM_CUDA(cudaStreamWaitEvent(us, c->ev_out, 0));
  SEM_CUDA(cudaStreamSynchronize(s));
  if (info) info->t_solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  t_err = cg_err;
  return cg;
}

sem_status sem_solve_host(sem_ctx* c, const double* f_host, double* u_host, sem_info* info, void* stream) {
  t_err.clear();
  NvtxScope nvtx_("sem_solve_host");
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  if (f_host == nullptr || u_host == nullptr) return fail(SEM_EINVAL, "null vector");
  const long long nn = c->g.Nx * c->g.Ny * c->g.Nz;
  const size_t bytes = sizeof(double) * (size_t)nn;
  cudaStream_t us = (cudaStream_t)stream;
  // the device copies are kept by the context (no allocation, and no
  // device-wide synchronization of a free, in the calls after the first)
  if (c->d_hf == nullptr && (dalloc(&c->d_hf, nn) != cudaSuccess || dalloc(&c->d_hu, nn) != cudaSuccess)) {
    if (c->d_hf) cudaFree(c->d_hf);
    c->d_hf = c->d_hu = nullptr;
    return fail(SEM_ENOMEM, "cannot allocate device fields");
  }
  double *df = c->d_hf, *du = c->d_hu;
  sem_status st = SEM_OK;
  cudaError_t e = cudaMemcpyAsync(df, f_host, bytes, cudaMemcpyHostToDevice, us);
  if (e != cudaSuccess) st = fail(SEM_ECUDA, cudaGetErrorString(e));
  if (st == SEM_OK) st = sem_solve(c, df, du, nullptr, info, stream);
  std::string keep = t_err;
  if (st == SEM_OK || st == SEM_ENOCONV || st == SEM_EBREAKDOWN) {
    e = cudaMemcpyAsync(u_host, du, bytes, cudaMemcpyDeviceToHost, us);
    if (e == cudaSuccess) e = cudaStreamSynchronize(us);
    if (e != cudaSuccess) {
      st = fail(SEM_ECUDA, cudaGetErrorString(e));
      keep = t_err;
    }
  }
  t_err = keep;
  return st;
}

sem_status sem_transform_skeleton(sem_ctx* c, const double* in, double* out, int kind, void* stream) {
  t_err.clear();
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  SEM_CHECK_VEC(in, double);
  SEM_CHECK_VEC(out, double);
  if (kind < 0 || kind > 3) return fail(SEM_EINVAL, "kind must be 0..3");
  static const int mat_of_kind[4] = {2, 1, 0, 3};
  launch_skel_transform(c->g, c->mat(mat_of_kind[kind]), in, out, (cudaStream_t)stream);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

sem_status sem_pack_skeleton(sem_ctx* c, const double* u_full, double* uB, void* stream) {
  t_err.clear();
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  SEM_CHECK_VEC(u_full, double);
  SEM_CHECK_VEC(uB, double);
  launch_pack(c->g, u_full, uB, (cudaStream_t)stream);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

sem_status sem_unpack_skeleton(sem_ctx* c, const double* uB, double* u_full, void* stream) {
  t_err.clear();
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  SEM_CHECK_VEC(uB, double);
  SEM_CHECK_VEC(u_full, double);
  launch_unpack(c->g, uB, u_full, 0, (cudaStream_t)stream);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

sem_status sem_profile_enable(sem_ctx* c, int enable) {
  t_err.clear();
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  c->prof = enable != 0;
  return SEM_OK;
}

sem_status sem_profile_read(sem_ctx* c, double* apply_ms, long long* apply_launches, int reset) {
  t_err.clear();
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  if (apply_ms) *apply_ms = c->prof_ms;
  if (apply_launches) *apply_launches = c->prof_count;
  if (reset) {
    c->prof_ms = 0.0;
    c->prof_count = 0;
  }
  return SEM_OK;
}

static sem_status ensure_adjoint(sem_ctx* c) {
  if (c->d_grad != nullptr) return SEM_OK;
  const SemGeom& g = c->g;
  const int q = g.p + 1;
  std::vector<double> h(c->hx);
  h.insert(h.end(), c->hy.begin(), c->hy.end());
  h.insert(h.end(), c->hz.begin(), c->hz.end());
  std::vector<double> kw(c->h1.K);
  kw.insert(kw.end(), c->h1.w.begin(), c->h1.w.end());
  bool ok = dalloc(&c->d_h, h.size()) == cudaSuccess && dalloc(&c->d_K, kw.size()) == cudaSuccess &&
            dalloc(&c->d_full, (size_t)(g.Nx * g.Ny * g.Nz)) == cudaSuccess &&
            dalloc(&c->d_E, (size_t)g.nelem * 5) == cudaSuccess &&
            dalloc(&c->d_grad, (size_t)(1 + g.mx + g.my + g.mz)) == cudaSuccess;
  if (!ok) return fail(SEM_ENOMEM, "cannot allocate adjoint buffers");
  SEM_CUDA(cudaMemcpy(c->d_h, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
  SEM_CUDA(cudaMemcpy(c->d_K, kw.data(), kw.size() * sizeof(double), cudaMemcpyHostToDevice));
  (void)q;
  return SEM_OK;
}

sem_status sem_solve_adjoint(sem_ctx* c, const double* gload, double* w, sem_info* info, void* stream) {
  t_err.clear();
  NvtxScope nvtx_("sem_solve_adjoint");
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  SEM_CHECK_VEC(gload, double);
  SEM_CHECK_VEC(w, double);
  sem_status st = ensure_adjoint(c);
  if (st != SEM_OK) return st;
  const SemGeom& g = c->g;
  const double *mx = c->d_mass, *my = mx + g.Nx, *mz = my + g.Ny;
  // sem_solve's load is (lumped mass) o f: pass f = g / m so that the load is g
  launch_mass_divide(g, mx, my, mz, gload, c->d_full, 0, (cudaStream_t)stream);
  SEM_CUDA(cudaGetLastError());
  return sem_solve(c, c->d_full, w, nullptr, info, stream);
}

sem_status sem_gradients(sem_ctx* c, const double* w, const double* u, const double* f, double* df,
                         double* dlambda, double* dhx, double* dhy, double* dhz, void* stream) {
  t_err.clear();
  NvtxScope nvtx_("sem_gradients");
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  SEM_CHECK_VEC(w, double);
  SEM_CHECK_VEC(u, double);
  SEM_CHECK_VEC(f, double);
  SEM_CHECK_VEC(df, double);
  sem_status st = ensure_adjoint(c);
  if (st != SEM_OK) return st;
  const SemGeom& g = c->g;
  cudaStream_t s = (cudaStream_t)stream;
  const double *mx = c->d_mass, *my = mx + g.Nx, *mz = my + g.Ny;
  const int q = g.p + 1;
  launch_mass_divide(g, mx, my, mz, w, df, 1, s);
  launch_lambda_gradient(g, mx, my, mz, w, u, c->d_partials, c->d_grad, &c->d_st->counter[3], s);
  launch_element_forms(g, c->d_K + q * q, c->d_K, w, u, f, c->d_E, s);
  const double* hx = c->d_h;
  const double* hy = hx + g.mx;
  const double* hz = hy + g.my;
  launch_width_gradient(g, 0, hx, hy, hz, c->lambda, c->d_E, c->d_grad + 1, s);
  launch_width_gradient(g, 1, hx, hy, hz, c->lambda, c->d_E, c->d_grad + 1 + g.mx, s);
  launch_width_gradient(g, 2, hx, hy, hz, c->lambda, c->d_E, c->d_grad + 1 + g.mx + g.my, s);
  SEM_CUDA(cudaGetLastError());
  std::vector<double> out(1 + g.mx + g.my + g.mz);
  SEM_CUDA(cudaMemcpyAsync(out.data(), c->d_grad, out.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  SEM_CUDA(cudaStreamSynchronize(s));
  if (dlambda) *dlambda = out[0];
  if (dhx) std::memcpy(dhx, out.data() + 1, g.mx * sizeof(double));
  if (dhy) std::memcpy(dhy, out.data() + 1 + g.mx, g.my * sizeof(double));
  if (dhz) std::memcpy(dhz, out.data() + 1 + g.mx + g.my, g.mz * sizeof(double));
  return SEM_OK;
}

sem_status sem_refine_history(const sem_ctx* c, double* rel_res, int capacity, int* count) {
  if (c == nullptr || count == nullptr || (capacity > 0 && rel_res == nullptr))
    return fail(SEM_EINVAL, "null argument");
  const int n = (int)c->refine_hist.size();
  *count = n;
  for (int i = 0; i < n && i < capacity; ++i) rel_res[i] = c->refine_hist[i];
  return SEM_OK;
}

long long sem_launch_count(void) { return sem_launch_total(); }

void sem_destroy(sem_ctx* c) { free_ctx(c); }

const char* sem_status_string(sem_status s) {
  switch (s) {
    case SEM_OK: return "ok";
    case SEM_EINVAL: return "invalid argument";
    case SEM_ENOMEM: return "out of memory";
    case SEM_ECUDA: return "CUDA error";
    case SEM_ENOCONV: return "not converged";
    case SEM_EBREAKDOWN: return "CG breakdown";
    case SEM_ENOTSUP: return "not supported";
  }
  return "unknown status";
}

const char* sem_last_error(void) { return t_err.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Condensed load without any allocation
// ---------------------------------------------------------------------------
// Scratch for sem_condense_rhs_noalloc: three element-interior work arrays of
// up to SEM_NOALLOC_MAX_CUBE doubles each (12 MiB in total).  The array is part
// of the library image: every GPU that loads the library holds it until the
// process exits.  Host code must not use its name as a device address; the
// address comes from cudaGetSymbolAddress, looked up once per device.
#define SEM_NOALLOC_MAX_CUBE (1LL << 19)
static __device__ __align__(256) double g_noalloc_scratch[3 * SEM_NOALLOC_MAX_CUBE];

namespace {
constexpr int kNoallocMaxDevices = 64;
double* g_noalloc_ptr[kNoallocMaxDevices] = {};
std::mutex g_noalloc_mu;

// Device address of g_noalloc_scratch on the current device (looked up on the
// first call per device).
sem_status noalloc_scratch(double** out) {
  int dev = 0;
  SEM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(SEM_EINVAL, "device index out of range for no-alloc scratch");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr)
      return fail(SEM_ECUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = static_cast<double*>(ptr);
  }
  *out = g_noalloc_ptr[dev];
  return SEM_OK;
}
}  // namespace

extern "C" sem_status sem_condense_rhs_noalloc(sem_ctx* c, const double* f, double* fB, sem_space space,
                                               void* stream) {
  t_err.clear();
  NvtxScope nvtx_("sem_condense_rhs_noalloc");
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  SEM_CHECK_VEC(f, double);
  SEM_CHECK_VEC(fB, double);
  if (space != SEM_SPACE_NODAL && space != SEM_SPACE_TRANSFORMED) return fail(SEM_EINVAL, "unknown space");
  const SemGeom& g = c->g;
  const long long cube = g.nelem * (long long)g.n * g.n * g.n;
  if (cube > SEM_NOALLOC_MAX_CUBE)
    return fail(SEM_EINVAL, "mesh too large for sem_condense_rhs_noalloc: elements * (p-1)^3 = " +
                                std::to_string(cube) + " exceeds " + std::to_string(SEM_NOALLOC_MAX_CUBE));
  double* scratch = nullptr;
  sem_status st = noalloc_scratch(&scratch);
  if (st != SEM_OK) return st;
  double* c0 = scratch;
  double* c1 = scratch + SEM_NOALLOC_MAX_CUBE;
  double* ft = scratch + 2 * SEM_NOALLOC_MAX_CUBE;
  cudaStream_t s = (cudaStream_t)stream;
  const double *mx = c->d_mass, *my = mx + g.Nx, *mz = my + g.Ny;
  // Every scratch entry that is read is written earlier in this call, and fB
  // is fully written before the face corrections are added: nothing has to be
  // cleared between calls.
  launch_load_skeleton(g, mx, my, mz, f, fB, s);
  launch_skel_transform(g, c->mat(0), fB, fB, s);
  launch_interior_load(g, mx, my, mz, f, c0, s);
  // FP64 mode products: the fixed scratch has no room for the per-element
  // scale exponents of the double-float form
  launch_mode(g, c->mat(0), 0, c0, c1, nullptr, s);
  launch_mode(g, c->mat(0), 1, c1, c0, nullptr, s);
  launch_mode(g, c->mat(0), 2, c0, ft, nullptr, s);
  launch_condense_faces(g, c->h1.basis, c->tab, ft, fB, s);
  if (space == SEM_SPACE_NODAL) launch_skel_transform(g, c->mat(3), fB, fB, s);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: CTA-tile shape of the operator kernel per (p, mesh, precision)
// ---------------------------------------------------------------------------
namespace {

using TuneKey = std::tuple<int, int, int, int, int>;   // p, mx, my, mz, element bytes
struct TuneResult {
  bool use_default;
  ApplyConfig cfg;
  double ms_default, ms_best;
};
std::map<TuneKey, TuneResult> g_tune_cache;
std::mutex g_tune_mu;

template <typename T>
sem_status time_apply(sem_ctx* c, const SemClassTables<T>& tab, const T* x, T* y, const ApplyConfig* cfg,
                      double* ms_out) {
  const SemGeom& g = c->g;
  cudaStream_t s = c->stream;
  cudaEvent_t e0, e1;
  SEM_CUDA(cudaEventCreate(&e0));
  SEM_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    SEM_CUDA(cudaMemsetAsync(y, 0, sizeof(T) * g.nb, s));
    SEM_CUDA(cudaEventRecord(e0, s));
    launch_tpt_apply<T>(g, c->h1.basis, tab, x, y, nullptr, nullptr, s, cfg);
    SEM_CUDA(cudaEventRecord(e1, s));
    SEM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    SEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0 && ms < best) best = ms;   // first launch is a warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SEM_CUDA(cudaGetLastError());
  *ms_out = best;
  return SEM_OK;
}

template <typename T>
sem_status tune_one(sem_ctx* c, const SemClassTables<T>& tab, const T* x, T* y, TuneResult* out) {
  const int n = c->g.n;
  double ms_def = 0.0;
  sem_status st = time_apply<T>(c, tab, x, y, nullptr, &ms_def);
  if (st != SEM_OK) return st;
  TuneResult r{true, ApplyConfig{}, ms_def, ms_def};
  auto consider = [&](const ApplyConfig& cfg) -> sem_status {
    if (!sem_apply_config_valid(n, sizeof(T), cfg)) return SEM_OK;
    double ms = 0.0;
    const sem_status s2 = time_apply<T>(c, tab, x, y, &cfg, &ms);
    if (s2 != SEM_OK) return s2;
    if (ms < r.ms_best) {
      r.ms_best = ms;
      r.use_default = false;
      r.cfg = cfg;
    }
    return SEM_OK;
  };
  // the other work mappings that exist for this degree and precision
  const int def = sem_apply_default_kind(n, sizeof(T));
  for (int kind : {kApplyWarp, kApplyPlane, kApplySlab, kApplyElement, kApplyRow, kApplyPencil}) {
    if (kind == def) continue;
    st = consider(sem_apply_config_kind(kind));
    if (st != SEM_OK) return st;
  }
  // CTA-tile shapes
  const int epbs[] = {1, 2, 3, 4, 5, 6, 8, 12, 16, 24, 32, 48, 64};
  const int kss[] = {n, (n + 1) / 2, (n + 3) / 4, 8, 4, 2};
  int tried = 0;
  for (int epb : epbs) {
    if (epb * n * n > 4096) continue;
    int last_ks = -1;
    for (int ks : kss) {
      if (ks < 1 || ks > n || ks == last_ks) continue;
      last_ks = ks;
      st = consider(sem_apply_config_make(n, sizeof(T), epb, ks));
      if (st != SEM_OK) return st;
      if (++tried >= 40) break;
    }
  }
  *out = r;
  return SEM_OK;
}

// Drops the instantiated graphs that hold an operator launch of one
// precision (the mixed loop trip holds both precisions' operators).
void drop_graph(sem_ctx* c, bool mixed) {
  cudaGraphExec_t& gr = mixed ? c->graph32 : c->graph;
  if (gr) {
    cudaGraphExecDestroy(gr);
    gr = nullptr;
  }
  if (c->graph32m) {
    cudaGraphExecDestroy(c->graph32m);
    c->graph32m = nullptr;
  }
}

}  // namespace

extern "C" sem_status sem_autotune(sem_ctx* c, double* ms_default, double* ms_best) {
  t_err.clear();
  NvtxScope nvtx_("sem_autotune");
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  const SemGeom& g = c->g;
  const bool mixed = c->opts.precision == SEM_PREC_MIXED;
  const TuneKey key{g.p, g.mx, g.my, g.mz, mixed ? 4 : 8};
  TuneResult r;
  bool have = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      r = it->second;
      have = true;
    }
  }
  if (!have) {
    sem_status st;
    if (mixed) {
      st = ensure_mixed(c);
      if (st != SEM_OK) return st;
      launch_cast_f32(g.nb, c->d_P, c->d_p32, c->stream);
      st = tune_one<float>(c, c->tab_f, c->d_p32, c->d_q32, &r);
    } else {
      st = tune_one<double>(c, c->tab, c->d_P, c->d_t2, &r);
    }
    if (st != SEM_OK) return st;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = r;
  }
  (mixed ? c->op32 : c->op64) = r.use_default ? ApplyConfig{} : r.cfg;
  drop_graph(c, mixed);
  if (!mixed) sync_deterministic(c);
  if (ms_default) *ms_default = r.ms_default;
  if (ms_best) *ms_best = r.ms_best;
  return SEM_OK;
}

extern "C" sem_status sem_set_operator_kernel(sem_ctx* c, int precision, int kind, int epb, int ks) {
  t_err.clear();
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  if (precision != SEM_PREC_FP64 && precision != SEM_PREC_MIXED)
    return fail(SEM_EINVAL, "precision must be SEM_PREC_FP64 or SEM_PREC_MIXED");
  const bool mixed = precision == SEM_PREC_MIXED;
  const size_t bytes = mixed ? 4 : 8;
  ApplyConfig cfg = kind == SEM_KERNEL_CTA_TILE ? sem_apply_config_make(c->g.n, bytes, epb, ks)
                                                : sem_apply_config_kind(kind);
  if (!sem_apply_config_valid(c->g.n, bytes, cfg))
    return fail(SEM_EINVAL, "operator kernel variant not available for this degree and precision");
  if (mixed) {
    const sem_status st = ensure_mixed(c);
    if (st != SEM_OK) return st;
  }
  (mixed ? c->op32 : c->op64) = cfg;
  drop_graph(c, mixed);
  return mixed ? SEM_OK : sync_deterministic(c);
}

extern "C" sem_status sem_check_vector(const sem_ctx* c, const void* p, int elem_bytes) {
  t_err.clear();
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  if (elem_bytes != 4 && elem_bytes != 8) return fail(SEM_EINVAL, "elem_bytes must be 4 or 8");
  return check_vec(c, p, (size_t)elem_bytes, "vector");
}

extern "C" sem_status sem_debug_oob(long long* count, long long* first) {
  t_err.clear();
  if (count == nullptr || first == nullptr) return fail(SEM_EINVAL, "null argument");
  *count = 0;
  *first = -1;
#ifdef SEM_DEBUG
  SEM_CUDA(cudaDeviceSynchronize());
  unsigned long long n = 0;
  long long f = -1;
  cudaError_t (*const take[])(unsigned long long*, long long*) = {sem_debug_take_kernels, sem_debug_take_apply,
                                                                 sem_debug_take_plane, sem_debug_take_slab,
                                                                 sem_debug_take_elem, sem_debug_take_row,
                                                                 sem_debug_take_pencil,
                                                                 sem_debug_take_compare};
  for (auto fn : take) SEM_CUDA(fn(&n, &f));
  *count = (long long)n;
  *first = n != 0 ? f : -1;
  return SEM_OK;
#else
  return fail(SEM_ENOTSUP, "the bounds record is compiled in debug builds only (SEM_DEBUG)");
#endif
}

extern "C" sem_status sem_debug_limit_skeleton(sem_ctx* c, long long bound) {
  t_err.clear();
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
#ifdef SEM_DEBUG
  if (bound < 0 || bound > c->g.nb) return fail(SEM_EINVAL, "bound must lie in [0, N_B]");
  c->g.dbg_bound = bound;
  return SEM_OK;
#else
  (void)bound;
  return fail(SEM_ENOTSUP, "the bounds record is compiled in debug builds only (SEM_DEBUG)");
#endif
}

extern "C" sem_status sem_debug_cg_step_timeout(sem_ctx* c, int* bar_fail, int* done) {
  t_err.clear();
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  if (bar_fail == nullptr || done == nullptr) return fail(SEM_EINVAL, "null argument");
#ifdef SEM_DEBUG
  sem_status st = ensure_mixed(c);
  if (st != SEM_OK) return st;
  if (!c->step_ok) return fail(SEM_ENOTSUP, "the device cannot run the one-pass CG step");
  const long long nb = c->g.nb;
  cudaStream_t s = c->stream;
  float* vecs[] = {c->d_x32, c->d_r32, c->d_p32, c->d_q32};
  for (float* v : vecs) SEM_CUDA(cudaMemsetAsync(v, 0, sizeof(float) * nb, s));
  // a running CG whose barrier count already holds every arrival it will get:
  // no CTA is the last to arrive, so every wait runs out
  PcgState h{};
  h.rho = 1.0;
  h.tol2 = 0.0;
  h.maxit = 1 << 30;
  h.bar_count = 2u * (unsigned)sem_num_sms();
  SEM_CUDA(cudaMemcpyAsync(c->d_st32, &h, sizeof(PcgState), cudaMemcpyHostToDevice, s));
  SEM_CUDA(launch_pcg_step<float>(nb, c->d_x32, c->d_r32, c->d_p32, c->d_q32, c->d_P32, c->d_partials, c->d_st32, s));
  SEM_CUDA(cudaMemcpyAsync(&h, c->d_st32, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  SEM_CUDA(cudaStreamSynchronize(s));
  *bar_fail = h.bar_fail;
  *done = h.done;
  SEM_CUDA(cudaMemsetAsync(c->d_st32, 0, sizeof(PcgState), s));   // a later solve starts from a clean record
  SEM_CUDA(cudaStreamSynchronize(s));
  return SEM_OK;
#else
  *bar_fail = 0;
  *done = 0;
  return fail(SEM_ENOTSUP, "the barrier test is compiled in debug builds only (SEM_DEBUG)");
#endif
}

extern "C" sem_status sem_get_operator_kernel(const sem_ctx* c, int precision, int* kind, int* epb, int* ks) {
  t_err.clear();
  if (c == nullptr || kind == nullptr) return fail(SEM_EINVAL, "null argument");
  if (precision != SEM_PREC_FP64 && precision != SEM_PREC_MIXED)
    return fail(SEM_EINVAL, "precision must be SEM_PREC_FP64 or SEM_PREC_MIXED");
  const bool mixed = precision == SEM_PREC_MIXED;
  const size_t bytes = mixed ? 4 : 8;
  const ApplyConfig& op = mixed ? c->op32 : c->op64;
  ApplyConfig eff = op.kind == kApplyAuto ? sem_apply_config_kind(sem_apply_default_kind(c->g.n, bytes)) : op;
  if (eff.kind == kApplyCta && op.kind == kApplyAuto) eff = sem_apply_config(c->g.n, bytes);
  *kind = eff.kind;
  if (epb) *epb = eff.kind == kApplyCta ? eff.epb : 0;
  if (ks) *ks = eff.kind == kApplyCta ? eff.ks : 0;
  return SEM_OK;
}

// ---------------------------------------------------------------------------
// Batched solves: one instantiated CUDA graph for many independent problems
// ---------------------------------------------------------------------------
namespace {

// One thread: keep looping while any problem is still iterating (and the
// safety cap on loop trips is not reached).
// A problem is still running while its flag is 0 (FP64: the CG state's
// `done`; mixed: the refinement control's `finished`).
__global__ void k_batch_decide(const int* const* flags, int count, int* trips, int cap,
                               cudaGraphConditionalHandle handle) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int active = 0;
  for (int i = 0; i < count; ++i) active |= (*flags[i] == 0);
  const int t = ++(*trips);
  cudaGraphSetConditional(handle, (active && t < cap) ? 1u : 0u);
}

}  // namespace

struct sem_batch {
  std::vector<sem_ctx*> ctxs;
  std::vector<const double*> f;
  std::vector<double*> u;
  std::vector<cudaStream_t> streams;   // [0] orchestrates, [1..count] one per problem
  std::vector<cudaEvent_t> events;
  int** d_flags = nullptr;
  int* d_trips = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long launches_fixed = 0, launches_per_trip = 0;
  int device = 0;
};

namespace {

void batch_free(sem_batch* b) {
  if (b == nullptr) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  if (b->d_flags) cudaFree(b->d_flags);
  if (b->d_trips) cudaFree(b->d_trips);
  delete b;
}

// Fork the problems onto their streams, run body(i, stream_i), join back.
template <typename F>
sem_status batch_fork_join(sem_batch* b, F body) {
  cudaStream_t s0 = b->streams[0];
  const int count = (int)b->ctxs.size();
  SEM_CUDA(cudaEventRecord(b->events[0], s0));
  for (int i = 0; i < count; ++i) {
    cudaStream_t si = b->streams[1 + i];
    SEM_CUDA(cudaStreamWaitEvent(si, b->events[0], 0));
    sem_status st = body(i, si);
    if (st != SEM_OK) return st;
    SEM_CUDA(cudaEventRecord(b->events[1 + i], si));
    SEM_CUDA(cudaStreamWaitEvent(s0, b->events[1 + i], 0));
  }
  return SEM_OK;
}

}  // namespace

extern "C" sem_status sem_batch_create(sem_ctx* const* ctxs, int count, const double* const* f, double* const* u,
                                       sem_batch** out) {
  t_err.clear();
  if (out == nullptr || ctxs == nullptr || f == nullptr || u == nullptr || count < 1)
    return fail(SEM_EINVAL, "null argument or empty batch");
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (check_ctx(ctxs[i]) != SEM_OK) return SEM_EINVAL;
    {
      const sem_ctx* c = ctxs[i];
      SEM_CHECK_VEC(f[i], double);
      SEM_CHECK_VEC(u[i], double);
    }
    if (ctxs[i]->opts.precision == SEM_PREC_MIXED && ctxs[i]->opts.mixed_scheme != 1)
      return fail(SEM_ENOTSUP, "batched mixed-precision solves use reliable updates (mixed_scheme 1)");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(SEM_EINVAL, "a context appears twice in the batch");
  }
  sem_batch* b = new sem_batch();
  cudaGetDevice(&b->device);
  b->ctxs.assign(ctxs, ctxs + count);
  b->f.assign(f, f + count);
  b->u.assign(u, u + count);
  auto bail = [&](sem_status st) {
    std::string keep = t_err;
    batch_free(b);
    t_err = keep;
    return st;
  };
  for (int i = 0; i <= count; ++i) {
    cudaStream_t st;
    cudaEvent_t ev;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
      return bail(fail(SEM_ECUDA, "cannot create batch streams"));
    b->streams.push_back(st);
    b->events.push_back(ev);
  }
  std::vector<int*> flags(count);
  int check = 1 << 30, cap = 0, refine_cap = 0;
  for (int i = 0; i < count; ++i) {
    sem_ctx* c = ctxs[i];
    sem_status st = ensure_cubes(c);
    if (st == SEM_OK && c->opts.precision == SEM_PREC_MIXED) st = ensure_ctl(c);
    if (st != SEM_OK) return bail(st);
    flags[i] = c->opts.precision == SEM_PREC_MIXED
                   ? reinterpret_cast<int*>(reinterpret_cast<char*>(c->d_ctl) + offsetof(MixedCtl, finished))
                   : reinterpret_cast<int*>(reinterpret_cast<char*>(c->d_st) + offsetof(PcgState, done));
    check = std::min(check, c->opts.check_every);
    cap = std::max(cap, c->opts.maxit);
    if (c->opts.precision == SEM_PREC_MIXED) refine_cap = std::max(refine_cap, c->opts.max_refine);
  }
  cap = cap / check + 2 + refine_cap;
  if (dalloc(&b->d_flags, count) != cudaSuccess || dalloc(&b->d_trips, 1) != cudaSuccess)
    return bail(fail(SEM_ENOMEM, "cannot allocate batch state"));
  if (cudaMemcpy(b->d_flags, flags.data(), count * sizeof(int*), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(fail(SEM_ECUDA, "cannot upload batch state"));
  cudaStream_t s0 = b->streams[0];
  cudaGraph_t pro = nullptr, epi = nullptr, main_g = nullptr;
  cudaError_t e;
  // prologue: condensed loads and CG initialisation, one branch per problem
  long long l0 = sem_launch_total();
  e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bail(fail(SEM_ECUDA, std::string("batch capture: ") + cudaGetErrorString(e)));
  sem_status cst = cudaMemsetAsync(b->d_trips, 0, sizeof(int), s0) == cudaSuccess ? SEM_OK : SEM_ECUDA;
  if (cst == SEM_OK)
    cst = batch_fork_join(b, [&](int i, cudaStream_t si) -> sem_status {
      sem_ctx* c = b->ctxs[i];
      const long long nb = c->g.nb;
      sem_status st = condense_rhs_t(c, b->f[i], c->d_b, si);
      if (st != SEM_OK) return st;
      if (c->opts.precision != SEM_PREC_MIXED) {
        launch_pcg_init<double>(nb, c->d_b, c->d_r, c->d_p, c->d_q, c->d_x, c->d_P, c->d_partials, c->d_st,
                                c->opts.rtol, c->opts.maxit, 0, si);
        return SEM_OK;
      }
      // mixed: x = 0, r = b in FP64, the FP32 CG on b32 = r, the refinement control
      return mixed_prologue(c, false, si);
    });
  e = cudaStreamEndCapture(s0, &pro);
  if (cst != SEM_OK || e != cudaSuccess) {
    if (pro) cudaGraphDestroy(pro);
    return bail(cst != SEM_OK ? cst : fail(SEM_ECUDA, std::string("batch prologue: ") + cudaGetErrorString(e)));
  }
  // epilogue: interior recovery
  e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
  cst = e == cudaSuccess ? batch_fork_join(b, [&](int i, cudaStream_t si) -> sem_status {
    sem_ctx* c = b->ctxs[i];
    if (c->opts.precision == SEM_PREC_MIXED) {   // whatever is not folded in yet (0 once folded)
      launch_pcg_flush<float>(c->g.nb, c->d_x32, c->d_p32, c->d_st32, si);
      launch_ir_update(c->g.nb, c->d_x, c->d_x32, 1.0, si);
    } else {
      launch_pcg_flush<double>(c->g.nb, c->d_x, c->d_p, c->d_st, si);
    }
    return recover_t(c, c->d_x, b->u[i], si);
  }) : SEM_ECUDA;
  e = cudaStreamEndCapture(s0, &epi);
  const long long l1 = sem_launch_total();
  if (cst != SEM_OK || e != cudaSuccess) {
    cudaGraphDestroy(pro);
    if (epi) cudaGraphDestroy(epi);
    return bail(cst != SEM_OK ? cst : fail(SEM_ECUDA, "batch epilogue capture failed"));
  }
  // main graph: prologue -> while(any problem iterating) { CG iterations } -> epilogue
  cudaGraphNode_t n_pro, n_loop, n_epi;
  cudaGraphConditionalHandle handle;
  e = cudaGraphCreate(&main_g, 0);
  if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&n_pro, main_g, nullptr, 0, pro);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, main_g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (e == cudaSuccess) e = cudaGraphAddNode(&n_loop, main_g, &n_pro, nullptr, 1, &cp);
  long long body_launches = 0;
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(s0, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const long long lb = sem_launch_total();
      cst = batch_fork_join(b, [&](int i, cudaStream_t si) -> sem_status {
        sem_ctx* c = b->ctxs[i];
        const SemGeom& g = c->g;
        if (c->opts.precision != SEM_PREC_MIXED) {
          for (int it = 0; it < check; ++it) {
            launch_tpt_apply<double>(g, c->h1.basis, c->tab, c->d_p, c->d_q, c->d_partials, c->d_st, si,
                                     &c->op64);
            launch_pcg_update<double>(g.nb, c->d_r, c->d_q, c->d_P, c->d_partials, c->d_st, si);
            launch_pcg_dir<double>(g.nb, c->d_x, c->d_r, c->d_p, c->d_q, c->d_P, c->d_st, si);
          }
          return SEM_OK;
        }
        // mixed: a refinement step when due, then FP32 CG iterations
        launch_mixed_step(g, c->h1.basis, c->tab, &c->op64, c->d_b, c->d_x, c->d_q, c->d_r, c->d_x32, c->d_r32,
                          c->d_p32, c->d_q32, c->d_P32, c->d_partials, c->d_ctl, c->d_st32, c->d_stg, si);
        for (int it = 0; it < check; ++it) {
          // batched problems run concurrently: the two-pass step (no grid barrier)
          const sem_status st = cg_iter_f32(c, si, nullptr, nullptr, false);
          if (st != SEM_OK) return st;
        }
        return SEM_OK;
      });
      k_batch_decide<<<1, 32, 0, s0>>>(b->d_flags, count, b->d_trips, cap, handle);
      sem_count_launch();
      body_launches = sem_launch_total() - lb;
      cudaGraph_t tmp = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(s0, &tmp);
      if (e2 != cudaSuccess) e = e2;
      if (cst != SEM_OK && e == cudaSuccess) e = cudaErrorUnknown;
    }
  }
  if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&n_epi, main_g, &n_loop, 1, epi);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, main_g, 0);
  cudaGraphDestroy(pro);
  cudaGraphDestroy(epi);
  if (main_g) cudaGraphDestroy(main_g);
  sem_count_launch(-(sem_launch_total() - l0));   // counted when the graph runs
  if (e != cudaSuccess) return bail(fail(SEM_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e)));
  b->launches_fixed = l1 - l0;
  b->launches_per_trip = body_launches;
  *out = b;
  return SEM_OK;
}

extern "C" sem_status sem_batch_solve(sem_batch* b, sem_info* infos, void* stream) {
  t_err.clear();
  NvtxScope nvtx_("sem_batch_solve");
  if (b == nullptr) return fail(SEM_EINVAL, "null batch");
  {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != b->device) {
      cudaGetLastError();
      return fail(SEM_EINVAL, "the current device is not the batch's device");
    }
  }
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t us = (cudaStream_t)stream;
  cudaStream_t s0 = b->streams[0];
  SEM_CUDA(cudaEventRecord(b->events[0], us));
  SEM_CUDA(cudaStreamWaitEvent(s0, b->events[0], 0));
  SEM_CUDA(cudaGraphLaunch(b->exec, s0));
  const int count = (int)b->ctxs.size();
  std::vector<PcgState> hs(count);
  std::vector<MixedCtl> hc(count);
  int trips = 0;
  for (int i = 0; i < count; ++i) {
    sem_ctx* c = b->ctxs[i];
    const bool mixed = c->opts.precision == SEM_PREC_MIXED;
    SEM_CUDA(cudaMemcpyAsync(&hs[i], mixed ? c->d_st32 : c->d_st, sizeof(PcgState), cudaMemcpyDeviceToHost, s0));
    if (mixed) SEM_CUDA(cudaMemcpyAsync(&hc[i], c->d_ctl, sizeof(MixedCtl), cudaMemcpyDeviceToHost, s0));
  }
  SEM_CUDA(cudaMemcpyAsync(&trips, b->d_trips, sizeof(int), cudaMemcpyDeviceToHost, s0));
  SEM_CUDA(cudaStreamSynchronize(s0));
  SEM_CUDA(cudaEventRecord(b->events[0], s0));
  SEM_CUDA(cudaStreamWaitEvent(us, b->events[0], 0));
  sem_count_launch(b->launches_fixed + (long long)trips * b->launches_per_trip);
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  sem_status worst = SEM_OK;
  for (int i = 0; i < count; ++i) {
    const PcgState& h = hs[i];
    sem_ctx* c = b->ctxs[i];
    sem_status st;
    double rel;
    int refinements = 0;
    if (c->opts.precision == SEM_PREC_MIXED) {
      const MixedCtl& m = hc[i];
      st = m.finished == 1 ? SEM_OK : (m.finished == 2 ? SEM_EBREAKDOWN : SEM_ENOCONV);
      refinements = m.refinements;
      const int last = std::min(refinements, kMixedHist - 1);
      rel = m.hist[last];
      c->refine_hist.assign(m.hist, m.hist + last + 1);
    } else {
      st = h.done == 1 ? SEM_OK : (h.done == 2 ? SEM_EBREAKDOWN : SEM_ENOCONV);
      rel = h.rr0 > 0 ? std::sqrt(h.rr / h.rr0) : 0.0;
    }
    if (infos) {
      infos[i].iters = h.iter;
      infos[i].refinements = refinements;
      infos[i].rel_res = rel;
      infos[i].t_solve_s = secs;
    }
    if (st != SEM_OK && worst == SEM_OK) worst = st;
  }
  if (worst != SEM_OK) return fail(worst, "at least one problem of the batch did not converge");
  return SEM_OK;
}

extern "C" void sem_batch_destroy(sem_batch* b) { batch_free(b); }

extern "C" sem_status sem_solve_batch(sem_ctx* const* ctxs, int count, const double* const* f, double* const* u,
                                      sem_info* infos, void* stream) {
  sem_batch* b = nullptr;
  sem_status st = sem_batch_create(ctxs, count, f, u, &b);
  if (st != SEM_OK) return st;
  st = sem_batch_solve(b, infos, stream);
  std::string keep = t_err;
  sem_batch_destroy(b);
  t_err = keep;
  return st;
}

// ---------------------------------------------------------------------------
// The paper's comparison variants: TPC and MMC operators, DC / BC / UC
// preconditioning (Sec. 5 and Sec. 8), on the nodal skeleton in FP64
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kMmcMaxBytes = 8ull << 30;   // the per-class dense face matrices MMC may hold

double* cmp_vec(sem_ctx* c, int k) { return c->d_cmp + (size_t)k * c->g.nb; }

sem_status ensure_cmp(sem_ctx* c) {
  if (c->d_cst != nullptr) return SEM_OK;
  const SemGeom& g = c->g;
  std::vector<double> kw(c->h1.K);
  kw.insert(kw.end(), c->h1.w.begin(), c->h1.w.end());
  if (dalloc(&c->d_cmpK, kw.size()) != cudaSuccess || dalloc(&c->d_cmp, 7 * (size_t)g.nb) != cudaSuccess ||
      dalloc(&c->d_cst, 1) != cudaSuccess)
    return fail(SEM_ENOMEM, "cannot allocate the comparison solver's vectors");
  SEM_CUDA(cudaMemcpy(c->d_cmpK, kw.data(), kw.size() * sizeof(double), cudaMemcpyHostToDevice));
  SEM_CUDA(cudaMemset(c->d_cst, 0, sizeof(CmpState)));
  return SEM_OK;
}

// Inverse diagonal of the nodal condensed operator (DC).
sem_status ensure_dc(sem_ctx* c, cudaStream_t s) {
  if (c->d_Pdc != nullptr) return SEM_OK;
  const SemGeom& g = c->g;
  const int ncls = g.ux * g.uy * g.uz;
  if (dalloc(&c->d_cdiag, (size_t)ncls * 6 * g.n * g.n) != cudaSuccess || dalloc(&c->d_Pdc, g.nb) != cudaSuccess)
    return fail(SEM_ENOMEM, "cannot allocate the nodal diagonal");
  double* diag = cmp_vec(c, 6);
  SEM_CUDA(cudaMemsetAsync(diag, 0, sizeof(double) * g.nb, s));
  launch_cmp_diag(g, c->h1.basis, c->tab, c->d_cmpK, c->d_cmpK + (g.p + 1) * (g.p + 1), c->mat(2), ncls, c->d_cdiag,
                  diag, s);
  launch_invert_diag(g, diag, c->d_Pdc, s);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

// Dense condensed face matrices of every width class and the elements of
// each class (MMC).
sem_status ensure_mmc(sem_ctx* c, cudaStream_t s) {
  if (c->d_mmc != nullptr) return SEM_OK;
  const SemGeom& g = c->g;
  const int ncls = g.ux * g.uy * g.uz;
  const long long M = 6LL * g.n * g.n;
  if ((size_t)ncls * M * M * sizeof(double) > kMmcMaxBytes)
    return fail(SEM_ENOTSUP, "MMC: the dense face matrices of this mesh exceed " +
                                 std::to_string(kMmcMaxBytes >> 30) + " GiB");
  std::vector<std::vector<int>> members(ncls);
  for (long long e = 0; e < g.nelem; ++e) {
    const int ex = (int)(e % g.mx), ey = (int)((e / g.mx) % g.my), ez = (int)(e / ((long long)g.mx * g.my));
    members[c->clsx[ex] + g.ux * (c->clsy[ey] + g.uy * c->clsz[ez])].push_back((int)e);
  }
  std::vector<int> flat;
  flat.reserve(g.nelem);
  c->cls_start.assign(ncls, 0);
  c->cls_count.assign(ncls, 0);
  int maxc = 0;
  for (int k = 0; k < ncls; ++k) {
    c->cls_start[k] = (long long)flat.size();
    c->cls_count[k] = (int)members[k].size();
    maxc = std::max(maxc, c->cls_count[k]);
    flat.insert(flat.end(), members[k].begin(), members[k].end());
  }
  if (dalloc(&c->d_mmc, (size_t)ncls * M * M) != cudaSuccess || dalloc(&c->d_cls_elems, flat.size()) != cudaSuccess ||
      dalloc(&c->d_mmcU, (size_t)maxc * M) != cudaSuccess || dalloc(&c->d_mmcY, (size_t)maxc * M) != cudaSuccess)
    return fail(SEM_ENOMEM, "cannot allocate the MMC face matrices");
  SEM_CUDA(cudaMemcpy(c->d_cls_elems, flat.data(), flat.size() * sizeof(int), cudaMemcpyHostToDevice));
  for (int k = 0; k < ncls; ++k) launch_mmc_build(g, c->h1.basis, c->tab, c->mat(2), k, c->d_mmc + (size_t)k * M * M, s);
  if (cublasCreate(&c->cublas) != CUBLAS_STATUS_SUCCESS) return fail(SEM_ECUDA, "cublasCreate failed");
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

// v = Hhat u on the nodal skeleton with operator variant op.
sem_status cmp_apply(sem_ctx* c, int op, const double* u, double* v, cudaStream_t s) {
  const SemGeom& g = c->g;
  const double* K = c->d_cmpK;
  const double* w = K + (g.p + 1) * (g.p + 1);
  if (op == SEM_OP_TPT) {
    launch_skel_transform(g, c->mat(2), u, c->d_t1, s);
    sem_status st = apply_t(c, c->d_t1, c->d_t2, s);
    if (st != SEM_OK) return st;
    launch_skel_transform(g, c->mat(3), c->d_t2, v, s);
    SEM_CUDA(cudaGetLastError());
    return SEM_OK;
  }
  SEM_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * g.nb, s));
  launch_tpc_apply(g, c->h1.basis, c->tab, K, w, c->mat(2), c->mat(3), u, v, op == SEM_OP_TPC ? 1 : 0, s);
  if (op == SEM_OP_MMC) {
    const int M = 6 * g.n * g.n;
    const double one = 1.0, zero = 0.0;
    if (cublasSetStream(c->cublas, s) != CUBLAS_STATUS_SUCCESS) return fail(SEM_ECUDA, "cublasSetStream failed");
    for (size_t k = 0; k < c->cls_count.size(); ++k) {
      const int cnt = c->cls_count[k];
      if (cnt == 0) continue;
      const int* el = c->d_cls_elems + c->cls_start[k];
      launch_mmc_gather(g, el, cnt, u, c->d_mmcU, s);
      if (cublasDgemm(c->cublas, CUBLAS_OP_N, CUBLAS_OP_N, M, cnt, M, &one, c->d_mmc + k * (size_t)M * M, M,
                      c->d_mmcU, M, &zero, c->d_mmcY, M) != CUBLAS_STATUS_SUCCESS)
        return fail(SEM_ECUDA, "cublasDgemm failed");
      launch_mmc_scatter(g, el, cnt, c->d_mmcY, v, s);
    }
  }
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

// z = M^-1 r with preconditioner pc (st: skip once the CG has stopped, may be null).
sem_status cmp_precond(sem_ctx* c, int pc, const double* r, double* z, const CmpState* st, cudaStream_t s) {
  const SemGeom& g = c->g;
  if (pc == SEM_PC_NONE) {
    launch_cmp_diagmul(g.nb, nullptr, r, z, st, s);
  } else if (pc == SEM_PC_DIAG) {
    launch_cmp_diagmul(g.nb, c->d_Pdc, r, z, st, s);
  } else {
    // block-Jacobi over faces, edges and vertices: T^T diag(T Ahat T^T)^-1 T (the blocks are diagonal in the
    // transformed system)
    double* t = cmp_vec(c, 6);
    launch_skel_transform(g, c->mat(0), r, t, s);
    launch_cmp_diagmul(g.nb, c->d_P, t, t, nullptr, s);
    launch_skel_transform(g, c->mat(1), t, z, s);
  }
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

sem_status check_variant(const sem_ctx* c, int op) {
  if (op != SEM_OP_TPT && op != SEM_OP_TPC && op != SEM_OP_MMC) return fail(SEM_EINVAL, "unknown operator variant");
  if (op != SEM_OP_TPT && c->g.p > kCmpMaxP)
    return fail(SEM_ENOTSUP, "TPC and MMC are built for p <= " + std::to_string(kCmpMaxP));
  return SEM_OK;
}

sem_status prepare_variant(sem_ctx* c, int op, cudaStream_t s) {
  sem_status st = ensure_cmp(c);
  if (st == SEM_OK && op == SEM_OP_MMC) st = ensure_mmc(c, s);
  return st;
}

}  // namespace

extern "C" sem_status sem_apply_condensed_variant(sem_ctx* c, int op, const double* uB, double* vB, void* stream) {
  t_err.clear();
  NvtxScope nvtx_("sem_apply_condensed_variant");
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  SEM_CHECK_VEC(uB, double);
  SEM_CHECK_VEC(vB, double);
  if (uB == vB) return fail(SEM_EINVAL, "uB and vB must not alias");
  sem_status st = check_variant(c, op);
  if (st != SEM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  st = prepare_variant(c, op, s);
  if (st != SEM_OK) return st;
  return cmp_apply(c, op, uB, vB, s);
}

extern "C" sem_status sem_diag_nodal(sem_ctx* c, double* diag, void* stream) {
  t_err.clear();
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  SEM_CHECK_VEC(diag, double);
  cudaStream_t s = (cudaStream_t)stream;
  sem_status st = ensure_cmp(c);
  if (st == SEM_OK) st = ensure_dc(c, s);
  if (st != SEM_OK) return st;
  // the diagonal is the inverse of the stored inverse (zero stays zero at Dirichlet entries)
  launch_invert_diag(c->g, c->d_Pdc, diag, s);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

extern "C" sem_status sem_solve_variant(sem_ctx* c, int op, int pc, const double* f, double* u, sem_info* info,
                                        void* stream) {
  t_err.clear();
  NvtxScope nvtx_("sem_solve_variant");
  if (check_ctx(c) != SEM_OK) return SEM_EINVAL;
  SEM_CHECK_VEC(f, double);
  SEM_CHECK_VEC(u, double);
  sem_status st = check_variant(c, op);
  if (st != SEM_OK) return st;
  if (pc != SEM_PC_NONE && pc != SEM_PC_DIAG && pc != SEM_PC_BLOCK) return fail(SEM_EINVAL, "unknown preconditioner");
  const auto t0 = std::chrono::steady_clock::now();
  if (info) std::memset(info, 0, sizeof(*info));
  cudaStream_t us = (cudaStream_t)stream;
  SEM_CUDA(cudaEventRecord(c->ev_in, us));
  SEM_CUDA(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
  cudaStream_t s = c->stream;
  st = prepare_variant(c, op, s);
  if (st == SEM_OK && pc == SEM_PC_DIAG) st = ensure_dc(c, s);
  if (st != SEM_OK) return st;
  const SemGeom& g = c->g;
  double *b = cmp_vec(c, 0), *x = cmp_vec(c, 1), *r = cmp_vec(c, 2), *p = cmp_vec(c, 3), *q = cmp_vec(c, 4),
         *z = cmp_vec(c, 5);
  // nodal condensed load (Algorithm 1), F~_I kept for the recovery
  st = condense_rhs_t(c, f, c->d_b, s);
  if (st != SEM_OK) return st;
  launch_skel_transform(g, c->mat(3), c->d_b, b, s);
  st = cmp_precond(c, pc, b, z, nullptr, s);
  if (st != SEM_OK) return st;
  launch_cmp_init(g.nb, b, x, r, z, p, c->d_partials, c->d_cst, c->opts.rtol, c->opts.maxit, s);
  CmpState& h = c->h_cst;
  // the stopping test is read after every iteration: the operators of this
  // loop cost milliseconds, the read a few microseconds, and no operator
  // runs past convergence
  for (int batch = 0; batch < c->opts.maxit + 2; ++batch) {
    SEM_CUDA(cudaMemcpyAsync(&h, c->d_cst, sizeof(CmpState), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    if (h.done != 0) break;
    {
      st = cmp_apply(c, op, p, q, s);
      if (st != SEM_OK) return st;
      launch_cmp_pq(g.nb, p, q, c->d_partials, c->d_cst, s);
      launch_cmp_xr(g.nb, x, r, p, q, c->d_partials, c->d_cst, s);
      st = cmp_precond(c, pc, r, z, c->d_cst, s);
      if (st != SEM_OK) return st;
      launch_cmp_rz(g.nb, r, z, c->d_partials, c->d_cst, s);
      launch_cmp_dir(g.nb, z, p, q, c->d_cst, s);
    }
  }
  SEM_CUDA(cudaMemcpyAsync(&h, c->d_cst, sizeof(CmpState), cudaMemcpyDeviceToHost, s));
  SEM_CUDA(cudaStreamSynchronize(s));
  // interior recovery from the nodal skeleton solution
  launch_skel_transform(g, c->mat(2), x, c->d_x, s);
  st = recover_t(c, c->d_x, u, s);
  if (st != SEM_OK) return st;
  SEM_CUDA(cudaEventRecord(c->ev_out, s));
  SEM_CUDA(cudaStreamWaitEvent(us, c->ev_out, 0));
  SEM_CUDA(cudaStreamSynchronize(s));
  if (info) {
    info->iters = h.iter;
    info->rel_res = h.rr0 > 0.0 ? std::sqrt(h.rr / h.rr0) : 0.0;
    info->t_solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (h.done == 2) return fail(SEM_EBREAKDOWN, "CG breakdown (p^T A p <= 0 or non-finite values)");
  if (h.done != 1) return fail(SEM_ENOCONV, "CG reached maxit without meeting rtol");
  return SEM_OK;
}
