// Internal declarations of the sm_103a condensed spectral-element library.
// Shared by the host setup, the kernels and the C-ABI layer; not installed.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#define SEM_MAXN 32   // interior nodes per direction, n = p - 1 <= 31

// Geometry of the Cartesian mesh and the packed skeleton layout (see sem.h).
struct SemGeom {
  int p, n, mx, my, mz;
  int ux, uy, uz;        // distinct element widths per axis (width classes)
  int slow;              // axis visited slowest by the operator kernel (most classes)
  long long nelem;
  long long off[8];      // block offsets: xf, yf, zf, xe, ye, ze, v, end(=N_B)
  long long nb;
#ifdef SEM_DEBUG
  long long dbg_bound;   // bound of the debug entity-offset checks (N_B unless lowered)
#endif
  long long Nx, Ny, Nz;  // global nodal grid
};

// Transformed 1D operators of Sec. 6 (passed by value to kernels).
//  lam   : eigenvalues Lambda of (K_II, M_II), ascending
//  k0, kp: K~_{I0} = S_II K_{I0}, K~_{Ip} = S_II K_{Ip}
//  Kss   : K~ corner entries [0][0], [0][p], [p][0], [p][p]
//  w0    : GLL end weight M_00 = M_pp
struct SemBasis {
  int n;
  double w0;
  double K[2][2];
  double lam[SEM_MAXN];
  double k[2][SEM_MAXN];
};

// Host-side 1D data computed at setup.
struct SemHost1D {
  int p;
  std::vector<double> x, w;          // GLL nodes and weights (p+1)
  std::vector<double> K;             // stiffness (p+1)^2 row-major
  std::vector<double> lam;           // n
  std::vector<double> V;             // n*n, V[r*n+c]: entry r of eigenvector c
  SemBasis basis;
};

// Per-element-width-class tables on the device.
template <typename T>
struct SemClassTables {
  const int* cls_x;   // [mx] class index of hx[ex]
  const int* cls_y;   // [my]
  const int* cls_z;   // [mz]
  const T* dcoef;     // [ncls][4] metric coefficients d0..d3
  const T* dinv;      // [ncls][n^3] D^-1, index (k n + j) n + i
  const T* coef;      // [ncls][coef_stride] operator coefficients (sem_apply.cu)
  long long coef_stride;
  const float* plane = nullptr;   // [ncls][plane_stride] blocks of the plane-per-lane FP32 kernel
  long long plane_stride = 0;     // (sem_apply_plane.cu); null where that kernel does not apply
  const T* coef_soa = nullptr;    // n = 1: coef transposed, entry r of class c at [r * ncls + c]
  int ncls = 0;                   // (the thread-per-element kernel); null for n > 1
  const float* plane_soa = nullptr;   // n = 2, 3: plane blocks transposed (the FP32 thread-per-element kernel)
};

// One class's coefficient block of the plane-per-lane FP32 operator (units of
// float; rows padded to rs = 4 ceil(n / 4), or 16 when n > 8, for 16-byte
// vector loads; padding entries are 0):
//   [pa, pa + rs)  a_i = d1 k_0[i]      [pb, pb + rs)  b_i = d1 k_1[i]
//   [pl1 .. pl3]   d1 lambda, d2 lambda, d3 lambda (one row each)
//   [pq, pq + 4n)  (c_m, d_m, e_m, g_m) = (d2 k_0, d2 k_1, d3 k_0, d3 k_1)[m]
//   [ps, ps + 36)  cO[6] = d_{dir+1} K~_{s,1-s}; face-diagonal constants[6]
//                  d0 w0 + d_{dir+1} K~_ss; edge-diagonal constants[12]
//                  w0 (d K~_ss + d' K~_s's'); vertex diagonals[8]; w0, w0^2, d0, 0
struct PlaneLayout {
  int rs, pa, pb, pl1, pl2, pl3, pq, ps, stride;
};
inline __host__ __device__ PlaneLayout plane_layout(int n) {
  PlaneLayout o;
  // rows of 16 for the two-chunk kernel (9 <= n <= 15), of 32 for the k-slab kernel (n >= 16)
  o.rs = n <= 8 ? (n + 3) & ~3 : (n <= 15 ? 16 : 32);
  o.pa = 0;
  o.pb = o.rs;
  o.pl1 = 2 * o.rs;
  o.pl2 = 3 * o.rs;
  o.pl3 = 4 * o.rs;
  o.pq = 5 * o.rs;
  o.ps = o.pq + 4 * n;
  o.stride = o.ps + 36;
  return o;
}
// Degrees served by the plane-per-lane kernels: n = p - 1 in [2, 15]
// (one row per lane for n <= 8, two half-rows per plane for 9 <= n <= 15).
inline __host__ __device__ bool plane_supported(int n) { return n >= 2 && n <= 15; }
// Degrees served by the k-slab kernel (sem_apply_slab.cu): 16 <= n <= 31.
inline __host__ __device__ bool slab_supported(int n) { return n >= 16 && n <= 31; }
// Degrees served by the FP32 thread-per-element kernel beyond n = 1
// (sem_apply_elem.cu): n = 2, 3.
inline __host__ __device__ bool elem_supported(int n) { return n == 2 || n == 3; }
// Whether the FP32 tables include the class blocks of plane_layout(n).
inline __host__ __device__ bool plane_table_used(int n) { return plane_supported(n) || slab_supported(n); }

// Offsets inside one class's operator coefficient block (units of T):
//   [0, 18n + 24): scaled line vectors and couplings, copied to shared memory
//       skd [3][2][n] = d_{dir+1} k_side        (condensed part)
//       skw [3][2][n] = d_{dir+1} w0 k_side     (lines inside a face)
//       skww[3][2][n] = d_{dir+1} w0^2 k_side   (lines along an edge)
//       cO[6], eO[6], vO[6] = d_{dir+1} {1, w0, w0^2} K~_{s,1-s}
//   fdiag [6][n^2]   diagonal of the primary part on the faces
//   ediag [12][n]    diagonal of the primary part on the edges
//   vdiag [8]        diagonal of the primary part at the vertices
//   ndinv [n^3]      -D^-1
struct CoefOffsets {
  int sm, fdiag, ediag, vdiag, ndinv;
  long long stride;
};
inline __host__ __device__ CoefOffsets coef_offsets(int n) {
  CoefOffsets o;
  o.sm = 18 * n + 24;
  o.fdiag = o.sm;
  o.ediag = o.fdiag + 6 * n * n;
  o.vdiag = o.ediag + 12 * n;
  o.ndinv = (o.vdiag + 8 + 3) & ~3;
  o.stride = ((long long)o.ndinv + (long long)n * n * n + 3) & ~3LL;
  return o;
}

// Device-resident CG scalars (one per solve in flight).
struct PcgState {
  double rho;        // r^T z of the current iterate
  double rho_new;
  double pq;         // p^T A p
  double rr;         // r^T r
  double rr0;        // b^T b, reference of the stopping rule
  double alpha, beta;
  double tol2;       // rtol^2 * rr0 (stop when rr <= tol2)
  double trig2;      // > 0: stop with done = 4 when rr <= trig2 (refinement trigger)
  int iter;          // iterations done
  int done;          // 1: converged, 2: breakdown, 3: maxit, 4: refinement triggered
  int maxit;
  int pad;
  unsigned int counter[4];  // last-block reduction tickets
  int xpend;                // 1: the last x += alpha p is still owed (the update stopped the CG)
  unsigned int flush_ticket;
  int pad2;
  unsigned int bar_count;   // grid barrier of the one-pass CG step: arrivals, generation
  unsigned int bar_gen;
  int bar_fail;             // 1: a barrier wait ran out (the CG stopped with done = 2)
  int pad3;
};

// Device-side control of one mixed-precision solve (FP32 CG with reliable
// updates inside FP64 refinement) replayed from a CUDA graph: the refinement
// kernels read `phase`, the loop decision reads `finished`.
constexpr int kMixedHist = 64;
struct MixedCtl {
  double bb;         // ||b||^2 of the FP64 condensed load
  double tol2;       // rtol^2 bb
  double delta2;     // reliable_delta^2
  double best;       // smallest relative FP64 residual so far
  double hist[kMixedHist];  // relative FP64 residual after each refinement step ([0]: start)
  int phase;         // 0: CG iterating, 1: refinement step due, 2: rebase the FP32 CG
  int finished;      // 0: running, 1: converged, 2: breakdown, 3: maxit, max_refine or stagnation
  int refinements, max_refine, stalls, restart;
  int xpend;         // the FP32 CG's owed x32 += alpha p32, taken over by the fold of this step
  unsigned int counter[2];
};

// ---- host helpers (sem_host.cpp) ----
bool sem_build_1d(int p, SemHost1D* out, std::string* err);

// ---- launch helpers (sem_kernels.cu) ----
void sem_count_launch(long long k = 1);
long long sem_launch_total();
