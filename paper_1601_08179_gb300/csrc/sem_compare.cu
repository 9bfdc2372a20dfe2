// The paper's comparison variants of the condensed operator and solver, on
// the nodal (untransformed) skeleton, FP64:
//
// * TPC (Sec. 5, Algorithm 3 with Table 1): primary part H_BB in nodal form
//   (Eq. east_east_primary_part: the face self blocks carry the dense K_II
//   along the face directions, 12 n^3 multiplications) plus the condensed
//   part through the interior eigenspace: the faces are mapped in with
//   V^T M_II along both face directions and the line vector V^T K_I0 normal to
//   the face, scaled by D^-1 (Eq. hii_diagonal), and mapped back with M_II V
//   and K_0I V (37 n^3).
// * MMC (Sec. 5, Algorithm 2): the same primary part plus the condensed part
//   as one dense 6n^2 x 6n^2 face-to-face matrix per width class, applied to
//   all elements of the class with one DGEMM (36 n^4 per element).
// * DC (Sec. 8): CG preconditioned with the inverse diagonal of the nodal
//   condensed operator; BC: with the exact inverse of its face, edge and
//   vertex self blocks, applied in tensor form (transform, diagonal of the
//   transformed operator, transform back: the blocks are diagonal in the
//   transformed system); UC: no preconditioner.
//
// These exist to compare against the transformed operator (TPT) and solver
// (BT) the library is built on; they are restricted to p <= 16.

#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "sem_device.cuh"
#include "sem_kernels.cuh"

using namespace semdev;

namespace {

constexpr int kCmpThreads = 256;

// Skeleton index of node (a, b, c) of element (ex, ey, ez), a, b, c in [0, p]
// with at least one on {0, p}; -1 for a node on the Dirichlet boundary.
__device__ __forceinline__ long long node_slot(const SemGeom& g, int ex, int ey, int ez, int a, int b, int c) {
  const int p = g.p, n = g.n;
  const bool na = a == 0 || a == p, nb = b == 0 || b == p, nc = c == 0 || c == p;
  bool dir = false;
  long long off;
  if (na + nb + nc == 1) {
    if (na) off = face_base(g, ex, ey, ez, a == p, &dir) + (long long)(c - 1) * n + (b - 1);
    else if (nb) off = face_base(g, ex, ey, ez, 2 + (b == p), &dir) + (long long)(c - 1) * n + (a - 1);
    else off = face_base(g, ex, ey, ez, 4 + (c == p), &dir) + (long long)(b - 1) * n + (a - 1);
  } else if (na + nb + nc == 2) {
    if (!na) off = edge_base(g, ex, ey, ez, (b == p) + 2 * (c == p), &dir) + (a - 1);
    else if (!nb) off = edge_base(g, ex, ey, ez, 4 + (a == p) + 2 * (c == p), &dir) + (b - 1);
    else off = edge_base(g, ex, ey, ez, 8 + (a == p) + 2 * (b == p), &dir) + (c - 1);
  } else {
    off = vert_index(g, ex, ey, ez, (a == p) + 2 * (b == p) + 4 * (c == p), &dir);
  }
  return dir ? -1 : off;
}

// Element node of face f (0 w, 1 e, 2 s, 3 n, 4 b, 5 t) at local (row, col):
// x-faces (row k, col j), y-faces (row k, col i), z-faces (row j, col i), all
// 0-based interior indices.
__device__ __forceinline__ void face_node(int f, int row, int col, int p, int* a, int* b, int* c) {
  const int d = f >> 1, s = (f & 1) ? p : 0;
  if (d == 0) { *a = s; *b = col + 1; *c = row + 1; }
  else if (d == 1) { *a = col + 1; *b = s; *c = row + 1; }
  else { *a = col + 1; *b = row + 1; *c = s; }
}

// Shared-memory plan of the TPC kernel (doubles): 1-D data, the element's
// nodal values with zero interior, transformed faces, a temporary, the cube,
// the condensed face outputs.
struct TpcSm {
  int K, w, A, B, u, F, T, cube, C, total;
};
__host__ __device__ inline TpcSm tpc_sm(int p) {
  const int q = p + 1, n = p - 1;
  TpcSm s;
  s.K = 0;
  s.w = s.K + q * q;
  s.A = s.w + q;
  s.B = s.A + n * n;
  s.u = s.B + n * n;
  s.F = s.u + q * q * q;
  s.T = s.F + 6 * n * n;
  s.cube = s.T + 6 * n * n;
  s.C = s.cube + n * n * n;
  s.total = s.C + 6 * n * n;
  return s;
}

// Nodal primary part at element node (a, b, c): (H_e u_e)(a, b, c) for the
// element's boundary values with zero interior (Eq. helmholtz_operator, the
// rightmost factor acting on x).  A line through the element interior meets
// the boundary at its two ends only.
__device__ __forceinline__ double tpc_primary(const double* K, const double* w, const double* ue, const double* d,
                                              int p, int a, int b, int c) {
  const int q = p + 1;
  const bool ia = a > 0 && a < p, ib = b > 0 && b < p, ic = c > 0 && c < p;
  const double* row = ue + ((long long)c * q + b) * q;
  double o = d[0] * w[a] * w[b] * w[c] * row[a];
  double sx = 0.0, sy = 0.0, sz = 0.0;
  if (ib && ic) {
    sx = K[a * q] * row[0] + K[a * q + p] * row[p];
  } else {
    for (int t = 0; t < q; ++t) sx = fma(K[a * q + t], row[t], sx);
  }
  if (ia && ic) {
    sy = K[b * q] * ue[(long long)c * q * q + a] + K[b * q + p] * ue[((long long)c * q + p) * q + a];
  } else {
    for (int t = 0; t < q; ++t) sy = fma(K[b * q + t], ue[((long long)c * q + t) * q + a], sy);
  }
  if (ia && ib) {
    sz = K[c * q] * ue[(long long)b * q + a] + K[c * q + p] * ue[((long long)p * q + b) * q + a];
  } else {
    for (int t = 0; t < q; ++t) sz = fma(K[c * q + t], ue[((long long)t * q + b) * q + a], sz);
  }
  o = fma(d[1] * w[b] * w[c], sx, o);
  o = fma(d[2] * w[a] * w[c], sy, o);
  o = fma(d[3] * w[a] * w[b], sz, o);
  return o;
}

// v += Hhat u on the nodal skeleton, one element per CTA iteration: the
// primary part always, the TPC condensed part when `condensed` (MMC adds its
// condensed part separately).  K: (p+1)^2 stiffness, w: GLL weights,
// A = V^T M_II, B = M_II V (row-major n x n).
__global__ void __launch_bounds__(kCmpThreads)
k_tpc_apply(SemGeom g, SemBasis bs, SemClassTables<double> tab, const double* __restrict__ Kg,
            const double* __restrict__ wg, const double* __restrict__ Ag, const double* __restrict__ Bg,
            const double* __restrict__ u, double* __restrict__ v, int condensed) {
  extern __shared__ double sh[];
  const int p = g.p, q = p + 1, n = g.n, n2 = n * n, q3 = q * q * q;
  const TpcSm L = tpc_sm(p);
  double *K = sh + L.K, *w = sh + L.w, *A = sh + L.A, *B = sh + L.B, *ue = sh + L.u;
  double *F = sh + L.F, *T = sh + L.T, *cube = sh + L.cube, *Cf = sh + L.C;
  __shared__ double d[4];
  for (int t = threadIdx.x; t < q * q; t += blockDim.x) K[t] = Kg[t];
  for (int t = threadIdx.x; t < q; t += blockDim.x) w[t] = wg[t];
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    A[t] = Ag[t];
    B[t] = Bg[t];
  }
  for (long long e = blockIdx.x; e < g.nelem; e += gridDim.x) {
    int ex, ey, ez;
    elem_coords(g, e, &ex, &ey, &ez);
    const int cls = elem_class(g, tab, ex, ey, ez);
    __syncthreads();   // the previous element is done with every buffer
    if (threadIdx.x < 4) d[threadIdx.x] = tab.dcoef[(long long)cls * 4 + threadIdx.x];
    // element nodal values, interior zero
    for (int t = threadIdx.x; t < q3; t += blockDim.x) {
      const int a = t % q, b = (t / q) % q, c = t / (q * q);
      double val = 0.0;
      if (a == 0 || a == p || b == 0 || b == p || c == 0 || c == p) {
        const long long s = node_slot(g, ex, ey, ez, a, b, c);
        if (s >= 0) val = u[s];
      }
      ue[t] = val;
    }
    __syncthreads();
    if (condensed) {
      // faces into the eigenspace directions along the face: F = A U A^T
      for (int t = threadIdx.x; t < 6 * n2; t += blockDim.x) {   // T = U A^T
        const int f = t / n2, r = (t % n2) / n, s = t % n;
        double acc = 0.0;
        for (int col = 0; col < n; ++col) {
          int a, b, c;
          face_node(f, r, col, p, &a, &b, &c);
          acc = fma(ue[((long long)c * q + b) * q + a], A[s * n + col], acc);
        }
        T[t] = acc;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < 6 * n2; t += blockDim.x) {   // F = A T
        const int f = t / n2, r = (t % n2) / n, s = t % n;
        double acc = 0.0;
        for (int rr = 0; rr < n; ++rr) acc = fma(A[r * n + rr], T[f * n2 + rr * n + s], acc);
        F[t] = acc;
      }
      __syncthreads();
      // expansion with the line vectors K~_I0, K~_Ip normal to each face, D^-1
      const double* dinv = tab.dinv + (long long)cls * n2 * n;
      for (int t = threadIdx.x; t < n2 * n; t += blockDim.x) {
        const int i = t % n, j = (t / n) % n, k = t / n2;
        double x = d[1] * (bs.k[0][i] * F[0 * n2 + k * n + j] + bs.k[1][i] * F[1 * n2 + k * n + j]);
        x = fma(d[2], bs.k[0][j] * F[2 * n2 + k * n + i] + bs.k[1][j] * F[3 * n2 + k * n + i], x);
        x = fma(d[3], bs.k[0][k] * F[4 * n2 + j * n + i] + bs.k[1][k] * F[5 * n2 + j * n + i], x);
        cube[t] = dinv[t] * x;
      }
      __syncthreads();
      // contraction onto each face with the same line vectors
      for (int t = threadIdx.x; t < 6 * n2; t += blockDim.x) {
        const int f = t / n2, r = (t % n2) / n, s = t % n, dr = f >> 1, side = f & 1;
        double acc = 0.0;
        for (int m = 0; m < n; ++m) {
          const int idx = dr == 0 ? (r * n + s) * n + m : dr == 1 ? (r * n + m) * n + s : (m * n + r) * n + s;
          acc = fma(bs.k[side][m], cube[idx], acc);
        }
        F[t] = d[dr + 1] * acc;
      }
      __syncthreads();
      // back to nodal face values: C = B F B^T
      for (int t = threadIdx.x; t < 6 * n2; t += blockDim.x) {   // T = F B^T
        const int f = t / n2, r = (t % n2) / n, s = t % n;
        double acc = 0.0;
        for (int col = 0; col < n; ++col) acc = fma(F[f * n2 + r * n + col], B[s * n + col], acc);
        T[t] = acc;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < 6 * n2; t += blockDim.x) {   // C = B T
        const int f = t / n2, r = (t % n2) / n, s = t % n;
        double acc = 0.0;
        for (int rr = 0; rr < n; ++rr) acc = fma(B[r * n + rr], T[f * n2 + rr * n + s], acc);
        Cf[t] = acc;
      }
      __syncthreads();
    }
    // outputs at every boundary node: primary - condensed (face nodes)
    for (int t = threadIdx.x; t < q3; t += blockDim.x) {
      const int a = t % q, b = (t / q) % q, c = t / (q * q);
      const bool na = a == 0 || a == p, nb = b == 0 || b == p, nc = c == 0 || c == p;
      if (!(na || nb || nc)) continue;
      const long long s = node_slot(g, ex, ey, ez, a, b, c);
      if (s < 0) continue;
      double o = tpc_primary(K, w, ue, d, p, a, b, c);
      if (condensed && na + nb + nc == 1) {
        int f, r, col;
        if (na) { f = a == p; r = c - 1; col = b - 1; }
        else if (nb) { f = 2 + (b == p); r = c - 1; col = a - 1; }
        else { f = 4 + (c == p); r = b - 1; col = a - 1; }
        o -= Cf[f * n2 + r * n + col];
      }
      atomicAdd(v + s, o);
    }
  }
}

// Row (f, r, c) of the face-to-eigenspace map of face f at cube point
// (i, j, k): the normal line vector times V^T M_II along both face directions
// (Table 1; without the metric factor).
__device__ __forceinline__ double mmc_g(const SemBasis& bs, const double* A, int n, int f, int r, int c, int i, int j,
                                        int k) {
  const int dr = f >> 1, side = f & 1;
  if (dr == 0) return bs.k[side][i] * A[k * n + r] * A[j * n + c];   // x-face (row k', col j')
  if (dr == 1) return bs.k[side][j] * A[k * n + r] * A[i * n + c];   // y-face (row k', col i')
  return bs.k[side][k] * A[j * n + r] * A[i * n + c];                // z-face (row j', col i')
}

// Dense condensed face-to-face matrix of width class `cls` (Algorithm 2):
// C[(f, r, c), (f', r', c')] = d_f d_f' sum_ijk G D^-1 G, stored with leading
// dimension 6 n^2 (symmetric).
__global__ void k_mmc_build(SemGeom g, SemBasis bs, SemClassTables<double> tab, const double* __restrict__ A, int cls,
                            double* __restrict__ C) {
  const int n = g.n, n2 = n * n, M = 6 * n2;
  const double* d = tab.dcoef + (long long)cls * 4;
  const double* dinv = tab.dinv + (long long)cls * n2 * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)M * M;
       t += (long long)gridDim.x * blockDim.x) {
    const int e1 = (int)(t / M), e2 = (int)(t % M);
    const int f1 = e1 / n2, r1 = (e1 % n2) / n, c1 = e1 % n;
    const int f2 = e2 / n2, r2 = (e2 % n2) / n, c2 = e2 % n;
    double acc = 0.0;
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
          acc = fma(mmc_g(bs, A, n, f1, r1, c1, i, j, k) * dinv[(k * n + j) * n + i],
                    mmc_g(bs, A, n, f2, r2, c2, i, j, k), acc);
    C[t] = d[1 + (f1 >> 1)] * d[1 + (f2 >> 1)] * acc;
  }
}

// Face values of the elements of one class into columns of U (6 n^2 rows,
// Dirichlet faces as zeros).
__global__ void k_mmc_gather(SemGeom g, const int* __restrict__ elems, int count, const double* __restrict__ u,
                             double* __restrict__ U) {
  const int n2 = g.n * g.n, M = 6 * n2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)count * M;
       t += (long long)gridDim.x * blockDim.x) {
    const long long col = t / M;
    const int row = (int)(t % M), f = row / n2;
    int ex, ey, ez;
    elem_coords(g, elems[col], &ex, &ey, &ez);
    bool dir = false;
    const long long base = face_base(g, ex, ey, ez, f, &dir);
    U[t] = dir ? 0.0 : u[base + row % n2];
  }
}

// v -= Y on the faces of the class's elements (the condensed part).
__global__ void k_mmc_scatter(SemGeom g, const int* __restrict__ elems, int count, const double* __restrict__ Y,
                              double* __restrict__ v) {
  const int n2 = g.n * g.n, M = 6 * n2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)count * M;
       t += (long long)gridDim.x * blockDim.x) {
    const long long col = t / M;
    const int row = (int)(t % M), f = row / n2;
    int ex, ey, ez;
    elem_coords(g, elems[col], &ex, &ey, &ez);
    bool dir = false;
    const long long base = face_base(g, ex, ey, ez, f, &dir);
    if (!dir) atomicAdd(v + base + row % n2, -Y[t]);
  }
}

// Diagonal of the condensed part of class `cls` on its face nodes:
// cd[f n^2 + r n + c] = d_f^2 sum_ijk G^2 D^-1.
__global__ void k_cmp_cdiag(SemGeom g, SemBasis bs, SemClassTables<double> tab, const double* __restrict__ A, int ncls,
                            double* __restrict__ cd) {
  const int n = g.n, n2 = n * n, M = 6 * n2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)ncls * M;
       t += (long long)gridDim.x * blockDim.x) {
    const int cls = (int)(t / M), e = (int)(t % M);
    const int f = e / n2, r = (e % n2) / n, c = e % n;
    const double* d = tab.dcoef + (long long)cls * 4;
    const double* dinv = tab.dinv + (long long)cls * n2 * n;
    double acc = 0.0;
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          const double gv = mmc_g(bs, A, n, f, r, c, i, j, k);
          acc = fma(gv * gv, dinv[(k * n + j) * n + i], acc);
        }
    cd[t] = d[1 + (f >> 1)] * d[1 + (f >> 1)] * acc;
  }
}

// Assembled diagonal of the nodal condensed operator: element by element the
// diagonal of the nodal primary part minus, on face nodes, the class's
// condensed diagonal; summed over the elements sharing a node.
__global__ void k_cmp_diag(SemGeom g, SemClassTables<double> tab, const double* __restrict__ K,
                           const double* __restrict__ w, const double* __restrict__ cd, double* __restrict__ diag) {
  const int p = g.p, q = p + 1, n = g.n, n2 = n * n, q3 = q * q * q;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.nelem * q3;
       t += (long long)gridDim.x * blockDim.x) {
    const long long e = t / q3;
    const int node = (int)(t % q3), a = node % q, b = (node / q) % q, c = node / (q * q);
    const bool na = a == 0 || a == p, nb = b == 0 || b == p, nc = c == 0 || c == p;
    if (!(na || nb || nc)) continue;
    int ex, ey, ez;
    elem_coords(g, e, &ex, &ey, &ez);
    const long long s = node_slot(g, ex, ey, ez, a, b, c);
    if (s < 0) continue;
    const int cls = elem_class(g, tab, ex, ey, ez);
    const double* d = tab.dcoef + (long long)cls * 4;
    double o = d[0] * w[a] * w[b] * w[c] + d[1] * w[b] * w[c] * K[a * q + a] + d[2] * w[a] * w[c] * K[b * q + b] +
               d[3] * w[a] * w[b] * K[c * q + c];
    if (na + nb + nc == 1) {
      int f, r, col;
      if (na) { f = a == p; r = c - 1; col = b - 1; }
      else if (nb) { f = 2 + (b == p); r = c - 1; col = a - 1; }
      else { f = 4 + (c == p); r = b - 1; col = a - 1; }
      o -= cd[(long long)cls * 6 * n2 + f * n2 + r * n + col];
    }
    atomicAdd(diag + s, o);
  }
}

// ---- CG on the nodal skeleton with any of the operators and preconditioners

__global__ void k_cmp_init(long long nb, const double* __restrict__ b, double* __restrict__ x, double* __restrict__ r,
                           const double* __restrict__ z, double* __restrict__ p, double* partials, CmpState* st,
                           double rtol, int maxit) {
  double rz = 0.0, rr = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
    rz = fma(b[i], z[i], rz);
    rr = fma(b[i], b[i], rr);
    x[i] = 0.0;
    r[i] = b[i];
    p[i] = z[i];
  }
  double v2[2] = {rz, rr}, tot[2];
  if (reduce_grid<2>(v2, partials, &st->counter[0], tot) && threadIdx.x == 0) {
    st->rho = tot[0];
    st->rr = st->rr0 = tot[1];
    st->tol2 = rtol * rtol * tot[1];
    st->iter = 0;
    st->maxit = maxit;
    st->done = (tot[1] <= st->tol2) ? 1 : (isfinite(tot[0]) && isfinite(tot[1]) ? 0 : 2);
  }
}

// alpha = rho / p^T q
__global__ void k_cmp_pq(long long nb, const double* __restrict__ p, const double* __restrict__ q, double* partials,
                         CmpState* st) {
  if (st->done) return;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x)
    s = fma(p[i], q[i], s);
  double v1[1] = {s}, tot[1];
  if (reduce_grid<1>(v1, partials, &st->counter[1], tot) && threadIdx.x == 0) {
    st->pq = tot[0];
    if (!(tot[0] > 0.0) || !isfinite(tot[0])) st->done = 2;
    else st->alpha = st->rho / tot[0];
  }
}

// x += alpha p, r -= alpha q; the stopping test on |r|
__global__ void k_cmp_xr(long long nb, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                         const double* __restrict__ q, double* partials, CmpState* st) {
  if (st->done) return;
  const double al = st->alpha;
  double rr = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
    x[i] = fma(al, p[i], x[i]);
    const double ri = fma(-al, q[i], r[i]);
    r[i] = ri;
    rr = fma(ri, ri, rr);
  }
  double v1[1] = {rr}, tot[1];
  if (reduce_grid<1>(v1, partials, &st->counter[2], tot) && threadIdx.x == 0) {
    st->rr = tot[0];
    st->iter += 1;
    if (!isfinite(tot[0])) st->done = 2;
    else if (tot[0] <= st->tol2) st->done = 1;
    else if (st->iter >= st->maxit) st->done = 3;
  }
}

// beta = r^T z / rho, p = z + beta p
__global__ void k_cmp_rz(long long nb, const double* __restrict__ r, const double* __restrict__ z, double* partials,
                         CmpState* st) {
  if (st->done) return;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x)
    s = fma(r[i], z[i], s);
  double v1[1] = {s}, tot[1];
  if (reduce_grid<1>(v1, partials, &st->counter[3], tot) && threadIdx.x == 0) {
    st->beta = tot[0] / st->rho;
    st->rho = tot[0];
  }
}

__global__ void k_cmp_dir(long long nb, const double* __restrict__ z, double* __restrict__ p, double* __restrict__ q,
                          const CmpState* st) {
  if (st->done) return;
  const double be = st->beta;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
    p[i] = fma(be, p[i], z[i]);
    q[i] = 0.0;
  }
}

// z = D r (D a diagonal; D null: z = r); skipped once the CG has stopped
__global__ void k_cmp_diagmul(long long nb, const double* __restrict__ D, const double* __restrict__ r,
                              double* __restrict__ z, const CmpState* st) {
  if (st != nullptr && st->done) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x)
    z[i] = D != nullptr ? D[i] * r[i] : r[i];
}

}  // namespace

static int cmp_grid(long long work, int per_block) {
  long long b = (work + per_block - 1) / per_block;
  const long long cap = (long long)sem_num_sms() * 32;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

void launch_tpc_apply(const SemGeom& g, const SemBasis& b, const SemClassTables<double>& t, const double* K,
                      const double* w, const double* A, const double* B, const double* u, double* v, int condensed,
                      cudaStream_t s) {
  const size_t smem = (size_t)tpc_sm(g.p).total * sizeof(double);
  static size_t attr = 0;
  if (smem > attr) {   // the first launch of each size happens outside any capture
    cudaFuncSetAttribute(k_tpc_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = smem;
  }
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tpc_apply, kCmpThreads, smem);
  long long grid = (long long)sem_num_sms() * (occ < 1 ? 1 : occ);
  if (grid > g.nelem) grid = g.nelem;
  k_tpc_apply<<<(int)grid, kCmpThreads, smem, s>>>(g, b, t, K, w, A, B, u, v, condensed);
  sem_count_launch();
}

void launch_mmc_build(const SemGeom& g, const SemBasis& b, const SemClassTables<double>& t, const double* A, int cls,
                      double* C, cudaStream_t s) {
  const long long M = 6LL * g.n * g.n;
  k_mmc_build<<<cmp_grid(M * M, kCmpThreads), kCmpThreads, 0, s>>>(g, b, t, A, cls, C);
  sem_count_launch();
}

void launch_mmc_gather(const SemGeom& g, const int* elems, int count, const double* u, double* U, cudaStream_t s) {
  const long long M = 6LL * g.n * g.n;
  k_mmc_gather<<<cmp_grid(M * count, kCmpThreads), kCmpThreads, 0, s>>>(g, elems, count, u, U);
  sem_count_launch();
}

void launch_mmc_scatter(const SemGeom& g, const int* elems, int count, const double* Y, double* v, cudaStream_t s) {
  const long long M = 6LL * g.n * g.n;
  k_mmc_scatter<<<cmp_grid(M * count, kCmpThreads), kCmpThreads, 0, s>>>(g, elems, count, Y, v);
  sem_count_launch();
}

void launch_cmp_diag(const SemGeom& g, const SemBasis& b, const SemClassTables<double>& t, const double* K,
                     const double* w, const double* A, int ncls, double* cd, double* diag, cudaStream_t s) {
  const long long M = 6LL * g.n * g.n;
  k_cmp_cdiag<<<cmp_grid(M * ncls, kCmpThreads), kCmpThreads, 0, s>>>(g, b, t, A, ncls, cd);
  const long long q3 = (long long)(g.p + 1) * (g.p + 1) * (g.p + 1);
  k_cmp_diag<<<cmp_grid(g.nelem * q3, kCmpThreads), kCmpThreads, 0, s>>>(g, t, K, w, cd, diag);
  sem_count_launch(2);
}

void launch_cmp_init(long long nb, const double* b, double* x, double* r, const double* z, double* p, double* partials,
                     CmpState* st, double rtol, int maxit, cudaStream_t s) {
  k_cmp_init<<<cmp_grid(nb, kCmpThreads * 4), kCmpThreads, 0, s>>>(nb, b, x, r, z, p, partials, st, rtol, maxit);
  sem_count_launch();
}

void launch_cmp_pq(long long nb, const double* p, const double* q, double* partials, CmpState* st, cudaStream_t s) {
  k_cmp_pq<<<cmp_grid(nb, kCmpThreads * 4), kCmpThreads, 0, s>>>(nb, p, q, partials, st);
  sem_count_launch();
}

void launch_cmp_xr(long long nb, double* x, double* r, const double* p, const double* q, double* partials,
                   CmpState* st, cudaStream_t s) {
  k_cmp_xr<<<cmp_grid(nb, kCmpThreads * 4), kCmpThreads, 0, s>>>(nb, x, r, p, q, partials, st);
  sem_count_launch();
}

void launch_cmp_rz(long long nb, const double* r, const double* z, double* partials, CmpState* st, cudaStream_t s) {
  k_cmp_rz<<<cmp_grid(nb, kCmpThreads * 4), kCmpThreads, 0, s>>>(nb, r, z, partials, st);
  sem_count_launch();
}

void launch_cmp_dir(long long nb, const double* z, double* p, double* q, const CmpState* st, cudaStream_t s) {
  k_cmp_dir<<<cmp_grid(nb, kCmpThreads * 4), kCmpThreads, 0, s>>>(nb, z, p, q, st);
  sem_count_launch();
}

void launch_cmp_diagmul(long long nb, const double* D, const double* r, double* z, const CmpState* st,
                        cudaStream_t s) {
  k_cmp_diagmul<<<cmp_grid(nb, kCmpThreads * 4), kCmpThreads, 0, s>>>(nb, D, r, z, st);
  sem_count_launch();
}

SEM_DEBUG_TU(compare)
