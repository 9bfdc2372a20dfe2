// sm_103a kernels of the statically condensed spectral-element Helmholtz solver:
// per-class tables, preconditioner, skeleton transforms, loads, recovery and
// the CG vector kernels.  The operator kernel itself is in sem_apply.cu:
//
// k_tpt_apply: the assembled transformed condensed operator
//   v~ = sum_e Rhat_e (H~_BB - H~_BI D^-1 H~_IB) Rhat_e^T u~
// evaluated element by element (Sec. 6):
//   * condensed part, Table 2: expand the six faces into the interior
//     eigenspace with d * K~_{I0} / K~_{Ip} (rank-1 per face and line), scale by
//     D^-1 (Eq. hii_diagonal), contract back with d * K~_{0I} / K~_{pI};
//     13 n^3 multiplications (Table 3);
//   * primary part H~_BB: the restriction of
//     H~ = d0 M~(x)M~(x)M~ + d1 M~(x)M~(x)K~ + d2 M~(x)K~(x)M~ + d3 K~(x)M~(x)M~
//     to the skeleton, with M~ = diag(w0, I, w0) and K~ = S K S^T, whose face
//     self-blocks are diagonal (Eq. east_east_primary_part_transformed); only
//     1D lines that lie in a face or an edge couple different entities;
//   * gather R^T and scatter-add R over faces (2 elements), edges (4) and
//     vertices (8) with FP64 reductions in L2 (red.global.add.f64).
// The per-element working set (faces, edges, vertices, a slab of the n^3
// eigenspace cube) lives in shared memory; nothing per element touches HBM
// except the skeleton values and the per-width-class D^-1 table (L2 resident).
#include <cuda_runtime.h>

#include <algorithm>

#include <atomic>
#include <cstdio>

#include "sem_device.cuh"
#include "sem_kernels.cuh"

using namespace semdev;

static std::atomic<long long> g_launches{0};
void sem_count_launch(long long k) { g_launches += k; }
long long sem_launch_total() { return g_launches.load(); }

namespace {

constexpr int kVecThreads = 256;
// Packs per thread per trip in the CG update and direction kernels, which run
// two 256-thread CTAs per SM (up to 128 registers: 4 vectors x 4 packs in
// flight per thread)
constexpr int kVecUnroll = 4;

// ---------------------------------------------------------------------------
// Per-width-class tables: d (Eq. metriccoeffelement) and D^-1 (Eq. hii_diagonal)
// ---------------------------------------------------------------------------
__global__ void k_class_tables(SemGeom g, SemBasis b, const double* __restrict__ wx,
                               const double* __restrict__ wy, const double* __restrict__ wz,
                               double lambda, double* __restrict__ dcoef, double* __restrict__ dinv) {
  const int n = g.n;
  const long long n3 = (long long)n * n * n;
  const long long ncls = (long long)g.ux * g.uy * g.uz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncls * (n3 + 4);
       t += (long long)gridDim.x * blockDim.x) {
    const long long c = t / (n3 + 4), r = t - c * (n3 + 4);
    const int cx = (int)(c % g.ux), cy = (int)((c / g.ux) % g.uy), cz = (int)(c / ((long long)g.ux * g.uy));
    const double h1 = wx[cx], h2 = wy[cy], h3 = wz[cz];
    const double J = h1 * h2 * h3 / 8.0;
    const double d0 = J * lambda, d1 = J * 4.0 / (h1 * h1), d2 = J * 4.0 / (h2 * h2), d3 = J * 4.0 / (h3 * h3);
    if (r < 4) {
      dcoef[c * 4 + r] = r == 0 ? d0 : (r == 1 ? d1 : (r == 2 ? d2 : d3));
    } else {
      const long long q = r - 4;
      const int i = (int)(q % n), j = (int)((q / n) % n), k = (int)(q / ((long long)n * n));
      dinv[c * n3 + q] = 1.0 / (d0 + d1 * b.lam[i] + d2 * b.lam[j] + d3 * b.lam[k]);
    }
  }
}

// ---------------------------------------------------------------------------
// Diagonal of the assembled transformed condensed operator (BT preconditioner)
// ---------------------------------------------------------------------------
// Face (dir, side) entry: d0 w0 + d K_ss + w0 (d' Lambda + d'' Lambda) (primary,
// Eq. east_east_primary_part_transformed) minus d^2 sum_t k_side[t]^2 D^-1 over
// the line into the interior (condensed self term).  Edge entry: the edge's
// primary diagonal (edges do not couple to the interior).  Vertex: primary.
__global__ void k_precond_diag(SemGeom g, SemBasis b, SemClassTables<double> tab, double* __restrict__ diag) {
  const int n = g.n, n2 = n * n;
  const int per = 6 * n2 + 12 * n + 8;
  const double w0 = b.w0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.nelem * per;
       t += (long long)gridDim.x * blockDim.x) {
    const long long e = t / per;
    const int r = (int)(t - e * per);
    int ex, ey, ez;
    elem_coords(g, e, &ex, &ey, &ez);
    const int c = elem_class(g, tab, ex, ey, ez);
    const double d[4] = {tab.dcoef[c * 4], tab.dcoef[c * 4 + 1], tab.dcoef[c * 4 + 2], tab.dcoef[c * 4 + 3]};
    const double* Dinv = tab.dinv + (long long)c * n2 * n;
    bool dir;
    long long gi;
    double val;
    if (r < 6 * n2) {
      const int slot = r / n2, idx = r - slot * n2, dd = slot >> 1, s = slot & 1;
      const int slow = idx / n, fast = idx - slow * n;
      gi = face_base(g, ex, ey, ez, slot, &dir) + idx;
      const double* ks = b.k[s];
      double cond = 0.0;
      if (dd == 0) {      // (j, k) = (fast, slow), line over i
        for (int i = 0; i < n; ++i) cond += ks[i] * ks[i] * Dinv[(slow * n + fast) * n + i];
        val = d[0] * w0 + d[1] * b.K[s][s] + w0 * (d[2] * b.lam[fast] + d[3] * b.lam[slow]) - d[1] * d[1] * cond;
      } else if (dd == 1) {  // (i, k), line over j
        for (int j = 0; j < n; ++j) cond += ks[j] * ks[j] * Dinv[(slow * n + j) * n + fast];
        val = d[0] * w0 + d[2] * b.K[s][s] + w0 * (d[1] * b.lam[fast] + d[3] * b.lam[slow]) - d[2] * d[2] * cond;
      } else {               // (i, j), line over k
        for (int k = 0; k < n; ++k) cond += ks[k] * ks[k] * Dinv[(k * n + slow) * n + fast];
        val = d[0] * w0 + d[3] * b.K[s][s] + w0 * (d[1] * b.lam[fast] + d[2] * b.lam[slow]) - d[3] * d[3] * cond;
      }
    } else if (r < 6 * n2 + 12 * n) {
      // an edge is shared by four elements: the one that sees it at its upper
      // sides (slot 4 grp + 3) sums all four shares in a fixed order
      const int q = r - 6 * n2, slot = q / n, l = q - slot * n;
      if ((slot & 3) != 3) continue;
      const int grp = slot >> 2;
      gi = edge_base(g, ex, ey, ez, slot, &dir) + l;
      if (dir) continue;
      // along-edge direction gets d w0^2 Lambda; the two transverse directions d w0 K_ss
      const int da = grp, t1 = grp == 0 ? 1 : 0, t2 = grp == 2 ? 1 : 2;
      val = 0.0;
      for (int nq = 0; nq < 4; ++nq) {
        const int s1 = nq & 1, s2 = nq >> 1;
        int nx = ex, ny = ey, nz = ez;
        if (grp == 0) { ny += 1 - s1; nz += 1 - s2; }
        else if (grp == 1) { nx += 1 - s1; nz += 1 - s2; }
        else { nx += 1 - s1; ny += 1 - s2; }
        const double* dn = tab.dcoef + elem_class(g, tab, nx, ny, nz) * 4;
        val += dn[0] * w0 * w0 + dn[da + 1] * w0 * w0 * b.lam[l] + dn[t1 + 1] * w0 * b.K[s1][s1] +
               dn[t2 + 1] * w0 * b.K[s2][s2];
      }
    } else {
      // a vertex is shared by eight elements: summed by the one that sees it
      // as its slot 7, in a fixed order
      const int slot = r - 6 * n2 - 12 * n;
      if (slot != 7) continue;
      gi = vert_index(g, ex, ey, ez, slot, &dir);
      if (dir) continue;
      val = 0.0;
      for (int nq = 0; nq < 8; ++nq) {
        const int sa = nq & 1, sb = (nq >> 1) & 1, sc = nq >> 2;
        const double* dn = tab.dcoef + elem_class(g, tab, ex + 1 - sa, ey + 1 - sb, ez + 1 - sc) * 4;
        val += dn[0] * w0 * w0 * w0 + w0 * w0 * (dn[1] * b.K[sa][sa] + dn[2] * b.K[sb][sb] + dn[3] * b.K[sc][sc]);
      }
    }
    // faces: two shares added onto zero (exact in either order); edges and
    // vertices: one add of the fixed-order sum
    if (!dir) atomicAdd(diag + gi, val);
  }
}

__global__ void k_invert_diag(long long nb, const double* __restrict__ diag, double* __restrict__ P) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
    const double d = diag[i];
    P[i] = d != 0.0 ? 1.0 / d : 0.0;
  }
}

// ---------------------------------------------------------------------------
// Skeleton transform: faces A U A^T, edges A u (in place allowed)
// ---------------------------------------------------------------------------
__global__ void k_skel_faces(SemGeom g, const double* __restrict__ A, const double* in, double* out, int fpb) {
  extern __shared__ double sh[];
  const int n = g.n, n2 = n * n;
  double* sA = sh;
  double* sU = sh + n2;            // [fpb][n2]
  double* sT = sU + fpb * n2;      // [fpb][n2]
  for (int t = threadIdx.x; t < n2; t += blockDim.x) sA[t] = A[t];
  const long long nfaces = (g.off[3] - g.off[0]) / n2;
  for (long long f0 = (long long)blockIdx.x * fpb; f0 < nfaces; f0 += (long long)gridDim.x * fpb) {
    __syncthreads();
    for (int t = threadIdx.x; t < fpb * n2; t += blockDim.x) {
      const long long f = f0 + t / n2;
      sU[t] = f < nfaces ? in[g.off[0] + f * n2 + (t % n2)] : 0.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < fpb * n2; t += blockDim.x) {   // T = U A^T
      const int fl = t / n2, r = t - fl * n2, row = r / n, col = r - row * n;
      const double* U = sU + fl * n2 + row * n;
      double s = 0.0;
      for (int c = 0; c < n; ++c) s = fma(U[c], sA[col * n + c], s);
      sT[t] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < fpb * n2; t += blockDim.x) {   // A T
      const int fl = t / n2, r = t - fl * n2, row = r / n, col = r - row * n;
      const long long f = f0 + fl;
      if (f >= nfaces) continue;
      const double* Tm = sT + fl * n2 + col;
      double s = 0.0;
      for (int c = 0; c < n; ++c) s = fma(sA[row * n + c], Tm[c * n], s);
      out[g.off[0] + f * n2 + r] = s;
    }
  }
}

__global__ void k_skel_edges(SemGeom g, const double* __restrict__ A, const double* in, double* out, int epb) {
  extern __shared__ double sh[];
  const int n = g.n;
  double* sA = sh;
  double* sU = sh + n * n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) sA[t] = A[t];
  const long long nedges = (g.off[6] - g.off[3]) / n;
  for (long long e0 = (long long)blockIdx.x * epb; e0 < nedges; e0 += (long long)gridDim.x * epb) {
    __syncthreads();
    for (int t = threadIdx.x; t < epb * n; t += blockDim.x) {
      const long long e = e0 + t / n;
      sU[t] = e < nedges ? in[g.off[3] + e * n + (t % n)] : 0.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < epb * n; t += blockDim.x) {
      const int el = t / n, row = t - el * n;
      const long long e = e0 + el;
      if (e >= nedges) continue;
      double s = 0.0;
      for (int c = 0; c < n; ++c) s = fma(sA[row * n + c], sU[el * n + c], s);
      out[g.off[3] + e * n + row] = s;
    }
  }
}

__global__ void k_copy_range(const double* in, double* out, long long a, long long b) {
  for (long long i = a + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < b; i += (long long)gridDim.x * blockDim.x)
    out[i] = in[i];
}

// ---------------------------------------------------------------------------
// Pack / unpack, lumped-mass loads, interior cubes
// ---------------------------------------------------------------------------
// Assembled lumped mass at a node factorises over the axes: m(gx) m(gy) m(gz)
// with m(g) = sum over the 1D elements containing g of (h_e / 2) w_local.
__global__ void k_pack(SemGeom g, const double* __restrict__ full, double* __restrict__ uB,
                       const double* __restrict__ mxs, const double* __restrict__ mys,
                       const double* __restrict__ mzs, int zero_dirichlet) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.nb; i += (long long)gridDim.x * blockDim.x) {
    long long gx, gy, gz;
    skel_node(g, i, &gx, &gy, &gz);
    double v = full[gx + g.Nx * (gy + g.Ny * gz)];
    if (mxs != nullptr) v *= mxs[gx] * mys[gy] * mzs[gz];
    if (zero_dirichlet && node_on_boundary(g, gx, gy, gz)) v = 0.0;
    uB[i] = v;
  }
}

__global__ void k_unpack(SemGeom g, const double* __restrict__ uB, double* __restrict__ full, int zero_dirichlet) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.nb; i += (long long)gridDim.x * blockDim.x) {
    long long gx, gy, gz;
    skel_node(g, i, &gx, &gy, &gz);
    const bool bnd = zero_dirichlet && node_on_boundary(g, gx, gy, gz);
    full[gx + g.Nx * (gy + g.Ny * gz)] = bnd ? 0.0 : uB[i];
  }
}

__global__ void k_interior_load(SemGeom g, const double* __restrict__ mxs, const double* __restrict__ mys,
                                const double* __restrict__ mzs, const double* __restrict__ f, double* __restrict__ X) {
  const int n = g.n, p = g.p;
  const long long n3 = (long long)n * n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.nelem * n3; t += (long long)gridDim.x * blockDim.x) {
    const long long e = t / n3;
    const long long r = t - e * n3;
    const int i = (int)(r % n), j = (int)((r / n) % n), k = (int)(r / ((long long)n * n));
    int ex, ey, ez;
    elem_coords(g, e, &ex, &ey, &ez);
    const long long gx = (long long)ex * p + i + 1, gy = (long long)ey * p + j + 1, gz = (long long)ez * p + k + 1;
    X[t] = mxs[gx] * mys[gy] * mzs[gz] * f[gx + g.Nx * (gy + g.Ny * gz)];
  }
}

__global__ void k_mode(SemGeom g, const double* __restrict__ A, int axis, const double* __restrict__ in,
                       double* __restrict__ out, double* __restrict__ grid) {
  __shared__ double sA[SEM_MAXN * SEM_MAXN];
  const int n = g.n, p = g.p;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) sA[t] = A[t];
  __syncthreads();
  const long long n3 = (long long)n * n * n;
  const int stride = axis == 0 ? 1 : (axis == 1 ? n : n * n);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.nelem * n3; t += (long long)gridDim.x * blockDim.x) {
    const long long e = t / n3;
    const long long r = t - e * n3;
    const int i = (int)(r % n), j = (int)((r / n) % n), k = (int)(r / ((long long)n * n));
    const int row = axis == 0 ? i : (axis == 1 ? j : k);
    const double* line = in + (t - (long long)row * stride);
    const double* Ar = sA + row * n;
    double s = 0.0;
    for (int c = 0; c < n; ++c) s = fma(Ar[c], line[(long long)c * stride], s);
    if (grid != nullptr) {
      int ex, ey, ez;
      elem_coords(g, e, &ex, &ey, &ez);
      const long long gx = (long long)ex * p + i + 1, gy = (long long)ey * p + j + 1, gz = (long long)ez * p + k + 1;
      grid[gx + g.Nx * (gy + g.Ny * gz)] = s;
    } else {
      out[t] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// Mode products in double-float arithmetic
// ---------------------------------------------------------------------------
// GB300's FP64 pipe runs at 1/64 of the FP32 pipe, and the O(n^4) mode
// products of load condensation and recovery (S (x) S (x) S on every interior
// cube, Algorithm 4) are bound by it in plain FP64.  They are computed here on
// the FP32 pipe in double-float form: a value is an unevaluated sum h + l of
// two floats (|l| <= ulp(h) / 2, 48 significant bits).  One multiply-add
// c += a b takes the exact product of the high parts (a product and its FMA
// residual), adds the cross terms a_h b_l + a_l b_h (the a_l b_l term, below
// 2^-48 of the product, is dropped), and adds the high product to the running
// sum with an error-free two-sum (Knuth), the rounding errors going to a
// second accumulator.  Explicit _rn intrinsics keep the compiler from fusing
// the error-free steps into FMAs.  Error of a length-n dot product: about
// n 2^-48 of sum |a b|, that of the FP64 FMA chain being n 2^-53.
// x 2^-shift = h + l: h the top 24 significant bits, l the next 24 (both
// truncated), formed from the bit fields with integer operations so that the
// split costs no FP64-pipe work; |x 2^-shift - h - l| < 2^-46 |x 2^-shift|.
// Values whose scaled parts would not both be normal floats
// (|x 2^-shift| < 2^-74 or >= 2^128), zeros and subnormals take the FP64
// conversion.
__device__ __forceinline__ float2 df_from_double(double x, int shift = 0) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const int ex0 = (int)((hi >> 20) & 0x7ffu), ex = ex0 - shift;
  if (ex0 == 0 || ex0 == 0x7ff || ex < 949 || ex > 1150) {
    const double xs = shift == 0 ? x : scalbn(x, -shift);
    const float h = __double2float_rn(xs);
    return make_float2(h, __double2float_rn(xs - (double)h));
  }
  const unsigned sign = hi & 0x80000000u;
  const unsigned long long mant = b & 0xfffffffffffffULL;                 // 52 bits below the leading 1
  const unsigned hb = sign | ((unsigned)(ex - 896) << 23) | (unsigned)(mant >> 29);
  const unsigned rem = (unsigned)(mant & 0x1fffffffULL);                   // the 29 bits h leaves out
  unsigned lb = 0u;
  if (rem != 0u) {
    const int pb = 31 - __clz((int)rem);                                   // leading bit of rem, 0..28
    const unsigned m = pb >= 23 ? (rem >> (pb - 23)) : (rem << (23 - pb));
    lb = sign | ((unsigned)(pb + ex - 948) << 23) | (m & 0x7fffffu);
  }
  return make_float2(__uint_as_float(hb), __uint_as_float(lb));
}

// f 2^e as a double, exactly, from the bit fields (integer operations);
// zeros directly, subnormals and results outside the normal double range
// through the FP64 path.
__device__ __forceinline__ double df_part_to_double(float f, int e) {
  const unsigned u = __float_as_uint(f);
  if ((u << 1) == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));   // +-0
  const int ex = (int)((u >> 23) & 0xffu), dex = ex + 896 + e;
  if (ex == 0 || ex == 0xff || dex <= 0 || dex >= 0x7ff) return scalbn((double)f, e);
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) | ((unsigned long long)dex << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}

// (s, e) += a b; s is the running sum of the high products, e collects the
// rounding errors and the low-order terms.
__device__ __forceinline__ void df_mac(float2 a, float2 b, float& s, float& e) {
  const float ph = __fmul_rn(a.x, b.x);
  float pl = __fmaf_rn(a.x, b.x, -ph);
  pl = __fmaf_rn(a.x, b.y, pl);
  pl = __fmaf_rn(a.y, b.x, pl);
  const float t = __fadd_rn(s, ph);
  const float bv = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bv)), __fsub_rn(ph, bv));
  s = t;
  e = __fadd_rn(e, __fadd_rn(err, pl));
}

// Double-float has the FP32 exponent range, so each element's cube is scaled
// by a power of two, 2^-shift with 2^shift <= max |x| < 2^(shift + 1), before
// the split (exact); the shift goes to eexp[e] and the last mode product
// scales back.  Entries below 2^-74 of their element's largest keep 24 to 48
// bits, which is below 2^-120 of that entry in absolute terms.  One CTA per
// element: the largest exponent, then the split (the second read hits L2).
__global__ void __launch_bounds__(256)
k_split_df(SemGeom g, const double* __restrict__ in, float2* __restrict__ out, int* __restrict__ eexp) {
  __shared__ int emax;
  const long long n3 = (long long)g.n * g.n * g.n;
  for (long long e = blockIdx.x; e < g.nelem; e += gridDim.x) {
    const double* x = in + e * n3;
    if (threadIdx.x == 0) emax = 0;
    __syncthreads();
    int m = 0;
    for (long long t = threadIdx.x; t < n3; t += blockDim.x) {
      const int ex = (int)(((unsigned long long)__double_as_longlong(x[t]) >> 52) & 0x7ffu);
      m = max(m, ex == 0x7ff ? 0 : ex);
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&emax, m);
    __syncthreads();
    // all zero or subnormal: scale the subnormals up as if the largest had exponent -1022
    const int shift = (emax == 0 ? 1 : emax) - 1023;
    for (long long t = threadIdx.x; t < n3; t += blockDim.x) out[e * n3 + t] = df_from_double(x[t], shift);
    if (threadIdx.x == 0) eexp[e] = shift;
    __syncthreads();
  }
}

// The same with one warp per element, for cubes of up to 4096 values (n <= 16).
__global__ void __launch_bounds__(256)
k_split_df_warp(SemGeom g, const double* __restrict__ in, float2* __restrict__ out, int* __restrict__ eexp) {
  const long long n3 = (long long)g.n * g.n * g.n;
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long e = w0; e < g.nelem; e += nw) {
    const double* x = in + e * n3;
    int m = 0;
    for (long long t = lane; t < n3; t += 32) {
      const int ex = (int)(((unsigned long long)__double_as_longlong(x[t]) >> 52) & 0x7ffu);
      m = max(m, ex == 0x7ff ? 0 : ex);
    }
    m = __reduce_max_sync(0xffffffffu, m);
    const int shift = (m == 0 ? 1 : m) - 1023;
    for (long long t = lane; t < n3; t += 32) out[e * n3 + t] = df_from_double(x[t], shift);
    if (lane == 0) eexp[e] = shift;
  }
}

// One mode product along `axis` (0: i, 1: j, 2: k) of all interior cubes:
// out[.. r ..] = sum_c A[r][c] in[.. c ..].  A thread takes one line of a cube
// along the axis and kModeRows consecutive rows r: each input value it loads
// serves kModeRows outputs, and the rows of A it reads are the same across
// the warp (shared-memory broadcast).  FINAL: the result is rounded to FP64
// into out, or into the interior nodes of the full nodal field when
// grid != nullptr, after scaling back by the element's 2^eexp[e]; otherwise
// it stays double-float and scaled.
constexpr int kModeRows = 8;

template <bool FINAL>
__global__ void __launch_bounds__(256)
k_mode_df(SemGeom g, const double* __restrict__ A, int axis, const float2* __restrict__ in, float2* __restrict__ out2,
          double* __restrict__ out, double* __restrict__ grid, const int* __restrict__ eexp) {
  __shared__ float2 sA[SEM_MAXN * SEM_MAXN];
  const int n = g.n, p = g.p, n2 = n * n;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) sA[t] = df_from_double(A[t]);
  __syncthreads();
  const long long n3 = (long long)n2 * n, nlines = g.nelem * n2;
  const int nrb = (n + kModeRows - 1) / kModeRows;
  const int stride = axis == 0 ? 1 : (axis == 1 ? n : n2);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nlines * nrb;
       t += (long long)gridDim.x * blockDim.x) {
    const int rb = (int)(t / nlines);
    const long long line = t - rb * nlines;
    const long long e = line / n2;
    const int q = (int)(line - e * n2), qa = q % n, qb = q / n;
    // the two coordinates across the line: (j, k), (i, k) or (i, j)
    const int i0 = axis == 0 ? 0 : qa, j0 = axis == 0 ? qa : (axis == 1 ? 0 : qb), k0 = axis == 2 ? 0 : qb;
    const long long base = e * n3 + i0 + (long long)n * (j0 + (long long)n * k0);
    const int r0 = rb * kModeRows;
    const float2* Arow[kModeRows];
#pragma unroll
    for (int u = 0; u < kModeRows; ++u) Arow[u] = sA + min(r0 + u, n - 1) * n;   // rows past n: computed, not stored
    float sh[kModeRows], sl[kModeRows];
#pragma unroll
    for (int u = 0; u < kModeRows; ++u) sh[u] = sl[u] = 0.f;
    for (int c = 0; c < n; ++c) {
      const float2 x = in[base + (long long)c * stride];
#pragma unroll
      for (int u = 0; u < kModeRows; ++u) df_mac(Arow[u][c], x, sh[u], sl[u]);
    }
#pragma unroll
    for (int u = 0; u < kModeRows; ++u) {
      const int r = r0 + u;
      if (r >= n) break;
      const long long o = base + (long long)r * stride;
      if (FINAL) {
        const int sc = eexp[e];
        const double v = df_part_to_double(sh[u], sc) + df_part_to_double(sl[u], sc);   // one FP64 addition
        if (grid != nullptr) {
          int ex, ey, ez;
          elem_coords(g, e, &ex, &ey, &ez);
          const int i = axis == 0 ? r : i0, j = axis == 1 ? r : j0, k = axis == 2 ? r : k0;
          const long long gx = (long long)ex * p + i + 1, gy = (long long)ey * p + j + 1,
                          gz = (long long)ez * p + k + 1;
          grid[gx + g.Nx * (gy + g.Ny * gz)] = v;
        } else {
          out[o] = v;
        }
      } else {
        const float h = __fadd_rn(sh[u], sl[u]);
        out2[o] = make_float2(h, __fsub_rn(sl[u], __fsub_rn(h, sh[u])));
      }
    }
  }
}

// fhat~ faces -= d k_side . (D^-1 Ft_I) along the line into the interior.
// One thread per face point: the shares of the two elements of the face are
// added in a fixed order (lower element first), so the condensed load does
// not depend on the order threads run in.
__global__ void k_condense_faces(SemGeom g, SemBasis b, SemClassTables<double> tab, const double* __restrict__ FtI,
                                 double* __restrict__ out) {
  const int n = g.n, n2 = n * n, mx = g.mx, my = g.my, mz = g.mz;
  const long long n3 = (long long)n2 * n;
  const long long nf0 = (long long)(mx + 1) * my * mz, nf1 = (long long)mx * (my + 1) * mz;
  const long long nf2 = (long long)mx * my * (mz + 1);
  const long long total = (nf0 + nf1 + nf2) * n2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    long long f = t / n2;
    const int idx = (int)(t - f * n2);
    int dd;
    if (f < nf0) dd = 0;
    else if (f < nf0 + nf1) { dd = 1; f -= nf0; }
    else { dd = 2; f -= nf0 + nf1; }
    int ex, ey, ez, pos, lim;   // pos: face position along dd (elements pos - 1 and pos)
    if (dd == 0) { pos = (int)(f % (mx + 1)); const long long q = f / (mx + 1); ey = (int)(q % my); ez = (int)(q / my); ex = pos; lim = mx; }
    else if (dd == 1) { ex = (int)(f % mx); const long long q = f / mx; pos = (int)(q % (my + 1)); ez = (int)(q / (my + 1)); ey = pos; lim = my; }
    else { ex = (int)(f % mx); const long long q = f / mx; ey = (int)(q % my); pos = (int)(q / my); ez = pos; lim = mz; }
    if (pos == 0 || pos == lim) continue;   // Dirichlet face
    bool dir = false;
    const long long gi = sem_dbg_entity(g.off[dd] + f * n2, n2, g, &dir) + idx;
    if (dir) continue;
    const int slow = idx / n, fast = idx - slow * n;
    long long off0, stride;
    if (dd == 0) { off0 = (long long)(slow * n + fast) * n; stride = 1; }
    else if (dd == 1) { off0 = (long long)slow * n2 + fast; stride = n; }
    else { off0 = (long long)slow * n + fast; stride = n2; }
    double sum = out[gi];
    for (int s = 1; s >= 0; --s) {   // the lower element sees the face at its side 1
      const int lx = ex - (dd == 0 ? s : 0), ly = ey - (dd == 1 ? s : 0), lz = ez - (dd == 2 ? s : 0);
      const long long e = lx + (long long)mx * (ly + (long long)my * lz);
      const int c = elem_class(g, tab, lx, ly, lz);
      const double* Dinv = tab.dinv + (long long)c * n3;
      const double* X = FtI + e * n3;
      const double* ks = b.k[s];
      double acc = 0.0;
      for (int m = 0; m < n; ++m) {
        const long long q = off0 + m * stride;
        acc = fma(ks[m], Dinv[q] * X[q], acc);
      }
      sum += -tab.dcoef[c * 4 + 1 + dd] * acc;
    }
    out[gi] = sum;
  }
}

// Z = D^-1 (Ft_I - H~_IB u~_B): expansion of the six faces (Table 2).
__global__ void k_recover_expand(SemGeom g, SemBasis b, SemClassTables<double> tab, const double* __restrict__ FtI,
                                 const double* __restrict__ uB, double* __restrict__ Z) {
  const int n = g.n, n2 = n * n;
  const long long n3 = (long long)n2 * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.nelem * n3; t += (long long)gridDim.x * blockDim.x) {
    const long long e = t / n3;
    const int r = (int)(t - e * n3);
    const int i = r % n, j = (r / n) % n, k = r / n2;
    int ex, ey, ez;
    elem_coords(g, e, &ex, &ey, &ez);
    const int c = elem_class(g, tab, ex, ey, ez);
    const double* d = tab.dcoef + c * 4;
    double acc = 0.0;
    for (int slot = 0; slot < 6; ++slot) {
      bool dir;
      const long long fb = face_base(g, ex, ey, ez, slot, &dir);
      if (dir) continue;
      const int dd = slot >> 1, s = slot & 1;
      double kv, uv;
      if (dd == 0) { kv = b.k[s][i]; uv = uB[fb + k * n + j]; }
      else if (dd == 1) { kv = b.k[s][j]; uv = uB[fb + k * n + i]; }
      else { kv = b.k[s][k]; uv = uB[fb + j * n + i]; }
      acc = fma(d[1 + dd] * kv, uv, acc);
    }
    Z[t] = tab.dinv[(long long)c * n3 + r] * (FtI[t] - acc);
  }
}

// ---------------------------------------------------------------------------
// CG vector kernels
// ---------------------------------------------------------------------------
// Per-thread partial sums are kept in T (FP32 for the inner solver, whose
// scalars need only FP32 accuracy) and combined across the grid in FP64.
// Vectors are accessed as 16-byte packs (float4 / double2) with a scalar tail.
template <typename T, int W>
struct alignas(sizeof(T) * W) Pack {
  T v[W];
};

// A preconditioner entry in the arithmetic type of its CG.
__device__ __forceinline__ double pval(double v) { return v; }
__device__ __forceinline__ float pval(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__global__ void __launch_bounds__(kVecThreads)
k_pcg_init(long long nb, const T* __restrict__ b, T* __restrict__ r, T* __restrict__ p,
           T* __restrict__ q, T* __restrict__ x, const prec_t<T>* __restrict__ P,
           double* __restrict__ partials, PcgState* st, double rtol, int maxit, int keep_x, int have_q) {
  T rz = T(0), rr = T(0), bb = T(0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
    const T bi = b[i];
    const T ri = have_q ? bi - q[i] : bi;
    const T zi = pval(P[i]) * ri;
    r[i] = ri;
    p[i] = zi;
    q[i] = T(0);
    if (!keep_x) x[i] = T(0);
    rz = fma(ri, zi, rz);
    rr = fma(ri, ri, rr);
    bb = fma(bi, bi, bb);
  }
  // the stopping rule is relative to ||b|| (= ||r_0|| for a zero start)
  double v[3] = {(double)rz, (double)rr, (double)bb}, tot[3];
  if (reduce_grid<3>(v, partials, &st->counter[1], tot) && threadIdx.x == 0) {
    st->rho = tot[0];
    st->rr = tot[1];
    st->rr0 = tot[2];
    st->tol2 = rtol * rtol * tot[2];
    st->iter = 0;
    st->maxit = maxit;
    st->alpha = st->beta = 0.0;
    st->trig2 = 0.0;
    st->xpend = 0;
    st->flush_ticket = 0u;
    st->bar_count = 0u;
    st->bar_fail = 0;
    if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) st->done = 2;
    else if (tot[1] <= st->tol2) st->done = 1;
    else st->done = 0;
  }
}

// r -= alpha q, rho' = r . P r, rr = r . r and the stopping tests.  The
// matching x += alpha p is done by k_pcg_dir (which reads p anyway); when
// this kernel stops the CG it is owed (st->xpend) and applied by
// k_pcg_flush or by the refinement fold.
template <typename T>
__global__ void __launch_bounds__(kVecThreads, 2)
k_pcg_update(long long nb, T* __restrict__ r, const T* __restrict__ q, const prec_t<T>* __restrict__ P,
             double* __restrict__ partials, PcgState* st) {
  if (st->done) return;
  constexpr int W = 16 / sizeof(T);
  using V = Pack<T, W>;
  using PV = Pack<prec_t<T>, W>;  // W preconditioner entries (8 bytes in BF16)
  const T alpha = (T)st->alpha;
  T rz = T(0), rr = T(0);
  const long long nv = nb / W;
  const long long g0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, gs = (long long)gridDim.x * blockDim.x;
  // kVecUnroll packs per thread per trip, all loads issued first (memory
  // latency, not bandwidth, bounds a one-pack loop)
  for (long long base = g0; base < nv; base += kVecUnroll * gs) {
    V rv[kVecUnroll], qv[kVecUnroll];
    PV Pv[kVecUnroll];
#pragma unroll
    for (int h = 0; h < kVecUnroll; ++h) {
      const long long iv = base + h * gs;
      if (iv < nv) {
        rv[h] = reinterpret_cast<const V*>(r)[iv];
        qv[h] = reinterpret_cast<const V*>(q)[iv];
        Pv[h] = reinterpret_cast<const PV*>(P)[iv];
      }
    }
#pragma unroll
    for (int h = 0; h < kVecUnroll; ++h) {
      const long long iv = base + h * gs;
      if (iv >= nv) break;
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const T ri = fma(-alpha, qv[h].v[c], rv[h].v[c]);
        rv[h].v[c] = ri;
        rz = fma(ri, pval(Pv[h].v[c]) * ri, rz);
        rr = fma(ri, ri, rr);
      }
      reinterpret_cast<V*>(r)[iv] = rv[h];
    }
  }
  for (long long i = nv * W + g0; i < nb; i += gs) {
    const T ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    rz = fma(ri, pval(P[i]) * ri, rz);
    rr = fma(ri, ri, rr);
  }
  double v[2] = {(double)rz, (double)rr}, tot[2];
  if (reduce_grid<2>(v, partials, &st->counter[2], tot) && threadIdx.x == 0) {
    const int it = st->iter + 1;
    st->iter = it;
    st->rho_new = tot[0];
    st->rr = tot[1];
    int done = 0;
    if (!isfinite(tot[0]) || !isfinite(tot[1])) {
      done = 2;
    } else if (tot[1] <= st->tol2) {
      done = 1;
    } else if (it >= st->maxit) {
      done = 3;
    } else if (st->trig2 > 0.0 && tot[1] <= st->trig2) {
      done = 4;              // refinement due: rho (of the previous residual) is kept
    } else {
      st->beta = tot[0] / st->rho;
      st->rho = tot[0];
    }
    st->xpend = done != 0 ? 1 : 0;
    st->done = done;
  }
}

// x += alpha p (the update of this iteration), then p = P r + beta p and q = 0.
template <typename T>
__global__ void __launch_bounds__(kVecThreads, 2)
k_pcg_dir(long long nb, T* __restrict__ x, const T* __restrict__ r, T* __restrict__ p, T* __restrict__ q,
          const prec_t<T>* __restrict__ P, PcgState* st) {
  if (st->done) return;
  constexpr int W = 16 / sizeof(T);
  using V = Pack<T, W>;
  using PV = Pack<prec_t<T>, W>;  // W preconditioner entries (8 bytes in BF16)
  const T alpha = (T)st->alpha, beta = (T)st->beta;
  const long long nv = nb / W;
  const long long g0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, gs = (long long)gridDim.x * blockDim.x;
  V zero;
#pragma unroll
  for (int c = 0; c < W; ++c) zero.v[c] = T(0);
  for (long long base = g0; base < nv; base += kVecUnroll * gs) {
    V xv[kVecUnroll], rv[kVecUnroll], pv[kVecUnroll];
    PV Pv[kVecUnroll];
#pragma unroll
    for (int h = 0; h < kVecUnroll; ++h) {
      const long long iv = base + h * gs;
      if (iv < nv) {
        xv[h] = reinterpret_cast<const V*>(x)[iv];
        rv[h] = reinterpret_cast<const V*>(r)[iv];
        Pv[h] = reinterpret_cast<const PV*>(P)[iv];
        pv[h] = reinterpret_cast<const V*>(p)[iv];
      }
    }
#pragma unroll
    for (int h = 0; h < kVecUnroll; ++h) {
      const long long iv = base + h * gs;
      if (iv >= nv) break;
#pragma unroll
      for (int c = 0; c < W; ++c) {
        xv[h].v[c] = fma(alpha, pv[h].v[c], xv[h].v[c]);
        pv[h].v[c] = fma(beta, pv[h].v[c], pval(Pv[h].v[c]) * rv[h].v[c]);
      }
      reinterpret_cast<V*>(x)[iv] = xv[h];
      reinterpret_cast<V*>(p)[iv] = pv[h];
      reinterpret_cast<V*>(q)[iv] = zero;
    }
  }
  for (long long i = nv * W + g0; i < nb; i += gs) {
    x[i] = fma(alpha, p[i], x[i]);
    p[i] = fma(beta, p[i], pval(P[i]) * r[i]);
    q[i] = T(0);
  }
}

// The owed x += alpha p of a CG that stopped in k_pcg_update (no-op
// otherwise); the last block clears the flag, so a second call adds nothing.
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
k_pcg_flush(long long nb, T* __restrict__ x, const T* __restrict__ p, PcgState* st) {
  if (!st->xpend) return;
  const T alpha = (T)st->alpha;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x)
    x[i] = fma(alpha, p[i], x[i]);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&st->flush_ticket, 1u) == gridDim.x - 1) {
      st->xpend = 0;
      st->flush_ticket = 0u;
    }
  }
}

// ---------------------------------------------------------------------------
// One-pass CG step: update and direction with a grid barrier between them
// ---------------------------------------------------------------------------
// After the operator (q = A p, alpha = rho / p.q) one CG step reads r, q, P,
// x and p once and writes r, x, p and q once: r -= alpha q, z = P r,
// rho' = r.z and rr = r.r, the stopping tests; then x += alpha p,
// p = z + beta p, q = 0.  beta needs rho' summed over the whole vector, so a
// grid barrier separates the two halves.  The grid is one CTA per SM,
// launched cooperatively (all CTAs resident); CTA b owns the contiguous packs
// [nv b / G, nv (b + 1) / G) and keeps their z in shared memory across the
// barrier (the launcher takes this kernel only when z fits).  Every CTA sums
// the per-CTA partials in the same
// order, so all take the same decision; CTA 0 records it.  The barrier's wait
// is bounded (about a second): on timeout the CTA records bar_fail, stops the
// CG with done = 2 and returns.
constexpr int kStepThreads = 768;
constexpr int kStepUnroll = 4;   // packs per thread per trip

constexpr long long kBarSpin = 1LL << 24;

// Grid barrier over st->bar_count / bar_gen (one use per launch; the last CTA
// to arrive resets the count).  Returns false in every thread of a CTA whose
// wait ran out.
static __device__ bool step_barrier(PcgState* st) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &st->bar_gen;
    const unsigned int g0 = *gen;
    __threadfence();
    int good = 1;
    if (atomicAdd(&st->bar_count, 1u) == gridDim.x - 1) {
      atomicExch(&st->bar_count, 0u);
      __threadfence();
      atomicAdd(&st->bar_gen, 1u);
    } else {
      long long spins = 0;
      while (*gen == g0) {
        if (++spins > kBarSpin) { good = 0; break; }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(kStepThreads, 1)
k_pcg_step(long long nb, T* __restrict__ x, T* __restrict__ r, T* __restrict__ p, T* __restrict__ q,
           const prec_t<T>* __restrict__ P, double* __restrict__ partials, PcgState* st) {
  extern __shared__ __align__(16) unsigned char step_smem[];
  __shared__ double tot_sh[2];
  __shared__ double red_sh[2 * 32];
  if (st->done) return;   // read by every CTA before the barrier; written after it
  constexpr int W = 16 / sizeof(T);
  using V = Pack<T, W>;
  using PV = Pack<prec_t<T>, W>;  // W preconditioner entries (8 bytes in BF16)
  V* zs = reinterpret_cast<V*>(step_smem);
  const T alpha = (T)st->alpha;
  const double rho = st->rho, tol2 = st->tol2, trig2 = st->trig2;
  const int it = st->iter + 1, maxit = st->maxit;
  const unsigned G = gridDim.x;
  const long long nv = nb / W;
  const long long c0 = nv * blockIdx.x / G, c1 = nv * (blockIdx.x + 1) / G;
  const bool tail_cta = blockIdx.x == G - 1;

  // ---- r -= alpha q, z = P r, partial dots.  Each thread issues the loads
  //      of kStepUnroll packs before using any (12 loads in flight): both
  //      halves are bound by memory latency, not by instruction issue
  T rz = T(0), rr = T(0);
  for (long long base = c0 + threadIdx.x; base < c1; base += kStepUnroll * kStepThreads) {
    V rv[kStepUnroll], qv[kStepUnroll];
    PV Pv[kStepUnroll];
#pragma unroll
    for (int h = 0; h < kStepUnroll; ++h) {
      const long long ih = base + (long long)h * kStepThreads;
      if (ih < c1) {
        rv[h] = reinterpret_cast<const V*>(r)[ih];
        qv[h] = reinterpret_cast<const V*>(q)[ih];
        Pv[h] = reinterpret_cast<const PV*>(P)[ih];
      }
    }
#pragma unroll
    for (int h = 0; h < kStepUnroll; ++h) {
      const long long ih = base + (long long)h * kStepThreads;
      if (ih >= c1) break;
      V zv;
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const T ri = fma(-alpha, qv[h].v[c], rv[h].v[c]);
        rv[h].v[c] = ri;
        zv.v[c] = pval(Pv[h].v[c]) * ri;
        rz = fma(ri, zv.v[c], rz);
        rr = fma(ri, ri, rr);
      }
      reinterpret_cast<V*>(r)[ih] = rv[h];
      zs[ih - c0] = zv;
    }
  }
  if (tail_cta) {
    for (long long i = nv * W + threadIdx.x; i < nb; i += kStepThreads) {
      const T ri = fma(-alpha, q[i], r[i]);
      r[i] = ri;
      rz = fma(ri, pval(P[i]) * ri, rz);
      rr = fma(ri, ri, rr);
    }
  }
  // the second half's first x and p packs do not depend on beta: their
  // loads are issued before the barrier and land while it is waited for
  V xv[kStepUnroll], pv[kStepUnroll];
#pragma unroll
  for (int h = 0; h < kStepUnroll; ++h) {
    const long long ih = c0 + threadIdx.x + (long long)h * kStepThreads;
    if (ih < c1) {
      xv[h] = reinterpret_cast<const V*>(x)[ih];
      pv[h] = reinterpret_cast<const V*>(p)[ih];
    }
  }
  double v[2] = {(double)rz, (double)rr};
  block_sum<2>(v, red_sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = v[0];
    partials[G + blockIdx.x] = v[1];
  }
  if (!step_barrier(st)) {
    // the CG stops as a breakdown whatever CTA 0 records after a late barrier
    // (its record is a compare-and-swap from 0)
    if (threadIdx.x == 0) {
      atomicExch(&st->bar_fail, 1);
      atomicExch(&st->done, 2);
    }
    return;
  }
  // ---- totals in a fixed order (the same in every CTA) and the decision
  if (threadIdx.x < 32) {
    double a = 0.0, b = 0.0;
    for (unsigned i = threadIdx.x; i < G; i += 32) {
      a += __ldcg(partials + i);
      b += __ldcg(partials + G + i);
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x == 0) {
      tot_sh[0] = a;
      tot_sh[1] = b;
    }
  }
  __syncthreads();
  const double RZ = tot_sh[0], RR = tot_sh[1];
  int done = 0;
  if (!isfinite(RZ) || !isfinite(RR)) done = 2;
  else if (RR <= tol2) done = 1;
  else if (it >= maxit) done = 3;
  else if (trig2 > 0.0 && RR <= trig2) done = 4;   // refinement due: rho (of the previous residual) is kept
  const double beta = done == 0 ? RZ / rho : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->iter = it;
    st->rho_new = RZ;
    st->rr = RR;
    if (done == 0) {
      st->beta = beta;
      st->rho = RZ;
    }
    st->xpend = done != 0 ? 1 : 0;   // a stopped CG owes x += alpha p (flush or refinement fold)
    atomicCAS(&st->done, 0, done);   // a CTA whose barrier wait ran out has already set 2
  }
  if (done != 0) return;
  // ---- x += alpha p, p = z + beta p, q = 0
  const T bt = (T)beta;
  V zero;
#pragma unroll
  for (int c = 0; c < W; ++c) zero.v[c] = T(0);
  for (long long base = c0 + threadIdx.x; base < c1; base += kStepUnroll * kStepThreads) {
    if (base != c0 + threadIdx.x) {   // the first trip's packs were loaded before the barrier
#pragma unroll
      for (int h = 0; h < kStepUnroll; ++h) {
        const long long ih = base + (long long)h * kStepThreads;
        if (ih < c1) {
          xv[h] = reinterpret_cast<const V*>(x)[ih];
          pv[h] = reinterpret_cast<const V*>(p)[ih];
        }
      }
    }
#pragma unroll
    for (int h = 0; h < kStepUnroll; ++h) {
      const long long ih = base + (long long)h * kStepThreads;
      if (ih >= c1) break;
      const V zv = zs[ih - c0];
#pragma unroll
      for (int c = 0; c < W; ++c) {
        xv[h].v[c] = fma(alpha, pv[h].v[c], xv[h].v[c]);
        pv[h].v[c] = fma(bt, pv[h].v[c], zv.v[c]);
      }
      reinterpret_cast<V*>(x)[ih] = xv[h];
      reinterpret_cast<V*>(p)[ih] = pv[h];
      reinterpret_cast<V*>(q)[ih] = zero;
    }
  }
  if (tail_cta) {
    for (long long i = nv * W + threadIdx.x; i < nb; i += kStepThreads) {
      x[i] = fma(alpha, p[i], x[i]);
      p[i] = fma(bt, p[i], pval(P[i]) * r[i]);
      q[i] = T(0);
    }
  }
}

// ---------------------------------------------------------------------------
// Iterative refinement (FP64 outer loop around the FP32 inner CG)
// ---------------------------------------------------------------------------
// r = b - Ax (FP64), rr = r.r -> st->rr; r32 = r * scale is written later.
__global__ void __launch_bounds__(kVecThreads)
k_ir_residual(long long nb, const double* __restrict__ b, const double* __restrict__ Ax, double* __restrict__ r,
              double* __restrict__ partials, PcgState* st) {
  double rr = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
    const double ri = b[i] - Ax[i];
    r[i] = ri;
    rr = fma(ri, ri, rr);
  }
  double v[1] = {rr}, tot[1];
  if (reduce_grid<1>(v, partials, &st->counter[3], tot) && threadIdx.x == 0) st->rr = tot[0];
}

// ---------------------------------------------------------------------------
// Device-side refinement control (mixed-precision solves replayed from a graph)
// ---------------------------------------------------------------------------
// One loop trip: gate -> fold -> FP64 operator -> residual + decision ->
// rebase -> direction, then FP32 CG iterations.  Each refinement kernel runs
// only in its phase; a finished problem runs none of them, and its FP32 CG
// state stays stopped (done != 0) so the CG kernels exit at once too.

// Start: after ||b||^2 (in st64->rr), the FP64 residual r_0 = b - A x_0 and
// the FP32 CG initialisation on b32 = r_0.  The FP32 CG stops at the global
// target rtol^2 ||b||^2.
__global__ void k_mixed_start(MixedCtl* ctl, const PcgState* st64, PcgState* st32, double rtol, double delta,
                              int max_refine) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double bb = st64->rr;
  ctl->bb = bb;
  ctl->tol2 = rtol * rtol * bb;
  ctl->delta2 = delta * delta;
  ctl->hist[0] = bb > 0.0 ? sqrt(st32->rr / bb) : 0.0;
  ctl->best = ctl->hist[0];
  st32->tol2 = ctl->tol2;
  ctl->phase = 0;
  ctl->refinements = 0;
  ctl->max_refine = max_refine;
  ctl->stalls = 0;
  ctl->restart = 0;
  ctl->counter[0] = ctl->counter[1] = 0u;
  if (!isfinite(bb) || !isfinite(st32->rr)) {
    ctl->finished = 2;
  } else if (bb == 0.0 || st32->rr <= ctl->tol2) {
    ctl->finished = 1;
  } else {
    ctl->finished = 0;
    st32->trig2 = ctl->delta2 * st32->rr;
  }
  if (ctl->finished != 0 && st32->done == 0) st32->done = 1;
}

// Top of a loop trip: a refinement step is due once the FP32 CG has stopped
// (triggered, converged in FP32, maxit or breakdown).  gate->done = 0 lets the
// FP64 operator run.
__global__ void k_mixed_gate(MixedCtl* ctl, PcgState* st32, PcgState* gate) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int d = st32->done;
  const bool refine = ctl->finished == 0 && d != 0;
  ctl->phase = refine ? 1 : 0;
  ctl->restart = d != 4;
  gate->done = refine ? 0 : 1;
  if (refine) {   // the fold applies the CG's owed x32 += alpha p32
    ctl->xpend = st32->xpend;
    st32->xpend = 0;
  }
}

// Phase 1: x += x32 (the FP32 correction, with the CG's owed alpha p32),
// x32 = 0, q = 0 (output of the FP64 operator).
__global__ void __launch_bounds__(kVecThreads)
k_mixed_fold(long long nb, double* __restrict__ x, float* __restrict__ x32, const float* __restrict__ p32,
             double* __restrict__ q, const MixedCtl* ctl, const PcgState* st32) {
  if (ctl->phase != 1) return;
  const float a = ctl->xpend ? (float)st32->alpha : 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
    x[i] += (double)fmaf(a, p32[i], x32[i]);
    x32[i] = 0.f;
    q[i] = 0.0;
  }
}

// Phase 1: r = b - A x in FP64 and the decision of the refinement step (the
// rules of the host-driven loop): converged, broken down, out of iterations or
// refinement steps, stalled (three steps without a 10 % gain), else rebase.
__global__ void __launch_bounds__(kVecThreads)
k_mixed_residual(long long nb, const double* __restrict__ b, const double* __restrict__ Ax, double* __restrict__ r,
                 double* __restrict__ partials, MixedCtl* ctl, const PcgState* st32) {
  if (ctl->phase != 1) return;
  double rr = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
    const double ri = b[i] - Ax[i];
    r[i] = ri;
    rr = fma(ri, ri, rr);
  }
  double v[1] = {rr}, tot[1];
  if (reduce_grid<1>(v, partials, &ctl->counter[0], tot) && threadIdx.x == 0) {
    const double rr_hi = tot[0];
    const int k = ++ctl->refinements;
    const double rel = ctl->bb > 0.0 ? sqrt(rr_hi / ctl->bb) : 0.0;
    ctl->hist[k < kMixedHist ? k : kMixedHist - 1] = rel;
    const int d = st32->done;
    if (!isfinite(rr_hi)) {
      ctl->finished = 2;
    } else if (rr_hi <= ctl->tol2) {
      ctl->finished = 1;
    } else if (d == 2) {
      ctl->finished = 2;
    } else if (d == 3 || k >= ctl->max_refine) {
      ctl->finished = 3;
    } else {
      ctl->stalls = rel < 0.9 * ctl->best ? 0 : ctl->stalls + 1;
      if (rel < ctl->best) ctl->best = rel;
      if (ctl->stalls >= 3) ctl->finished = 3;
      else ctl->phase = 2;
    }
  }
}

// Phase 2: the FP32 CG continues from the true residual (residual
// replacement): r32 = r, rho' = r32 . P r32, beta = rho' / rho (0 when the
// direction restarts), rr, the next trigger delta^2 rr, done = 0.
__global__ void __launch_bounds__(kVecThreads)
k_mixed_rebase(long long nb, const double* __restrict__ r, const prec_t<float>* __restrict__ P, float* __restrict__ r32,
               double* __restrict__ partials, MixedCtl* ctl, PcgState* st32) {
  if (ctl->phase != 2) return;
  float rz = 0.f, rr = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
    const float ri = (float)r[i];
    r32[i] = ri;
    rz = fmaf(ri, pval(P[i]) * ri, rz);
    rr = fmaf(ri, ri, rr);
  }
  double v[2] = {(double)rz, (double)rr}, tot[2];
  if (reduce_grid<2>(v, partials, &ctl->counter[1], tot) && threadIdx.x == 0) {
    st32->beta = ctl->restart ? 0.0 : tot[0] / st32->rho;
    st32->rho = tot[0];
    st32->rr = tot[1];
    st32->trig2 = ctl->delta2 * tot[1];
    st32->done = (isfinite(tot[0]) && isfinite(tot[1])) ? 0 : 2;
  }
}

// Phase 2: p = P r32 + beta p, q = 0 (the direction step of the replaced residual).
__global__ void __launch_bounds__(kVecThreads)
k_mixed_dir(long long nb, const float* __restrict__ r32, float* __restrict__ p, float* __restrict__ q,
            const prec_t<float>* __restrict__ P, const MixedCtl* ctl, const PcgState* st32) {
  if (ctl->phase != 2 || st32->done != 0) return;
  const float beta = (float)st32->beta;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
    p[i] = fmaf(beta, p[i], pval(P[i]) * r32[i]);
    q[i] = 0.f;
  }
}

__global__ void k_to_prec32(long long nb, const double* __restrict__ in, prec_t<float>* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x)
    out[i] = __double2bfloat16(in[i]);
}

__global__ void k_scale_to_f32(long long nb, const double* __restrict__ in, double scale, float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)(in[i] * scale);
}

// x += scale * (double) c
__global__ void k_ir_update(long long nb, double* __restrict__ x, const float* __restrict__ c, double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x)
    x[i] = fma(scale, (double)c[i], x[i]);
}

int g_num_sms = 0;
int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 152;
  }
  return g_num_sms;
}

int grid_for(long long work, int threads, int per_sm = 8) {
  long long b = (work + threads - 1) / threads;
  long long cap = (long long)num_sms() * per_sm;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

int sem_num_sms() { return num_sms(); }

int sem_vec_blocks() { return num_sms() * 4; }

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
void launch_cast_f32(long long n, const double* in, float* out, cudaStream_t s) {
  k_scale_to_f32<<<grid_for(n, 256), 256, 0, s>>>(n, in, 1.0, out);
  sem_count_launch();
}

void launch_cast_prec32(long long n, const double* in, prec_t<float>* out, cudaStream_t s) {
  k_to_prec32<<<grid_for(n, 256), 256, 0, s>>>(n, in, out);
  sem_count_launch();
}

void launch_class_tables(const SemGeom& g, const SemBasis& b, const double* ux_w, const double* uy_w,
                         const double* uz_w, double lambda, double* dcoef, double* dinv, cudaStream_t s) {
  const long long ncls = (long long)g.ux * g.uy * g.uz;
  const long long work = ncls * ((long long)g.n * g.n * g.n + 4);
  k_class_tables<<<grid_for(work, 256, 16), 256, 0, s>>>(g, b, ux_w, uy_w, uz_w, lambda, dcoef, dinv);
  sem_count_launch();
}

void launch_precond_diag(const SemGeom& g, const SemBasis& b, const SemClassTables<double>& t, double* diag,
                         cudaStream_t s) {
  const long long work = g.nelem * (6LL * g.n * g.n + 12LL * g.n + 8);
  k_precond_diag<<<grid_for(work, 256, 16), 256, 0, s>>>(g, b, t, diag);
  sem_count_launch();
}

void launch_invert_diag(const SemGeom& g, const double* diag, double* P, cudaStream_t s) {
  k_invert_diag<<<grid_for(g.nb, 256), 256, 0, s>>>(g.nb, diag, P);
  sem_count_launch();
}

void launch_skel_transform(const SemGeom& g, const double* A, const double* in, double* out, cudaStream_t s) {
  const int n = g.n, n2 = n * n;
  const long long nfaces = (g.off[3] - g.off[0]) / n2;
  int fpb = 256 / n2;
  if (fpb < 1) fpb = 1;
  size_t smf = (size_t)(n2 + 2 * fpb * n2) * sizeof(double);
  k_skel_faces<<<grid_for(nfaces, fpb, 16), 256, smf, s>>>(g, A, in, out, fpb);
  const long long nedges = (g.off[6] - g.off[3]) / n;
  int epb = 256 / n;
  if (epb < 1) epb = 1;
  size_t sme = (size_t)(n2 + epb * n) * sizeof(double);
  k_skel_edges<<<grid_for(nedges, epb, 16), 256, sme, s>>>(g, A, in, out, epb);
  sem_count_launch(2);
  if (in != out) {
    k_copy_range<<<grid_for(g.nb - g.off[6], 256), 256, 0, s>>>(in, out, g.off[6], g.nb);
    sem_count_launch();
  }
}

void launch_load_skeleton(const SemGeom& g, const double* mxs, const double* mys, const double* mzs,
                          const double* f, double* out, cudaStream_t s) {
  k_pack<<<grid_for(g.nb, 256), 256, 0, s>>>(g, f, out, mxs, mys, mzs, 1);
  sem_count_launch();
}

void launch_interior_load(const SemGeom& g, const double* mxs, const double* mys, const double* mzs,
                          const double* f, double* X, cudaStream_t s) {
  const long long work = g.nelem * (long long)g.n * g.n * g.n;
  k_interior_load<<<grid_for(work, 256, 16), 256, 0, s>>>(g, mxs, mys, mzs, f, X);
  sem_count_launch();
}

void launch_mode(const SemGeom& g, const double* A, int axis, const double* in, double* out, double* grid,
                 cudaStream_t s) {
  const long long work = g.nelem * (long long)g.n * g.n * g.n;
  k_mode<<<grid_for(work, 256, 16), 256, 0, s>>>(g, A, axis, in, out, grid);
  sem_count_launch();
}

void launch_mode3(const SemGeom& g, const double* A, double* in, double* tmp, int* eexp, double* out, double* grid,
                  cudaStream_t s) {
  const long long lines = g.nelem * (long long)g.n * g.n * ((g.n + kModeRows - 1) / kModeRows);
  const int mblocks = grid_for(lines, 256, 16);
  const int sblocks = (int)std::min<long long>(g.nelem, (long long)num_sms() * 16);
  // a double-float value takes the 8 bytes of the FP64 one it replaces
  float2* a = reinterpret_cast<float2*>(tmp);
  float2* b = reinterpret_cast<float2*>(in);
  if ((long long)g.n * g.n * g.n <= 4096)
    k_split_df_warp<<<grid_for(g.nelem * 32, 256, 16), 256, 0, s>>>(g, in, a, eexp);
  else
    k_split_df<<<sblocks, 256, 0, s>>>(g, in, a, eexp);
  k_mode_df<false><<<mblocks, 256, 0, s>>>(g, A, 0, a, b, nullptr, nullptr, eexp);
  k_mode_df<false><<<mblocks, 256, 0, s>>>(g, A, 1, b, a, nullptr, nullptr, eexp);
  k_mode_df<true><<<mblocks, 256, 0, s>>>(g, A, 2, a, nullptr, out, grid, eexp);
  sem_count_launch(4);
}

void launch_condense_faces(const SemGeom& g, const SemBasis& b, const SemClassTables<double>& t,
                           const double* FtI, double* out, cudaStream_t s) {
  const long long faces = (long long)(g.mx + 1) * g.my * g.mz + (long long)g.mx * (g.my + 1) * g.mz +
                          (long long)g.mx * g.my * (g.mz + 1);
  const long long work = faces * g.n * g.n;
  k_condense_faces<<<grid_for(work, 256, 16), 256, 0, s>>>(g, b, t, FtI, out);
  sem_count_launch();
}

void launch_recover_expand(const SemGeom& g, const SemBasis& b, const SemClassTables<double>& t,
                           const double* FtI, const double* uB, double* Z, cudaStream_t s) {
  const long long work = g.nelem * (long long)g.n * g.n * g.n;
  k_recover_expand<<<grid_for(work, 256, 16), 256, 0, s>>>(g, b, t, FtI, uB, Z);
  sem_count_launch();
}

void launch_pack(const SemGeom& g, const double* full, double* uB, cudaStream_t s) {
  k_pack<<<grid_for(g.nb, 256), 256, 0, s>>>(g, full, uB, nullptr, nullptr, nullptr, 0);
  sem_count_launch();
}

void launch_unpack(const SemGeom& g, const double* uB, double* full, int zero_dirichlet, cudaStream_t s) {
  k_unpack<<<grid_for(g.nb, 256), 256, 0, s>>>(g, uB, full, zero_dirichlet);
  sem_count_launch();
}

template <typename T>
void launch_pcg_init(long long nb, const T* b, T* r, T* p, T* q, T* x, const prec_t<T>* P, double* partials,
                     PcgState* st, double rtol, int maxit, int keep_x, cudaStream_t s) {
  k_pcg_init<T><<<sem_vec_blocks(), kVecThreads, 0, s>>>(nb, b, r, p, q, x, P, partials, st, rtol, maxit, keep_x,
                                                         keep_x);
  sem_count_launch();
}

void launch_mixed_start(MixedCtl* ctl, const PcgState* st64, PcgState* st32, double rtol, double delta,
                        int max_refine, cudaStream_t s) {
  k_mixed_start<<<1, 32, 0, s>>>(ctl, st64, st32, rtol, delta, max_refine);
  sem_count_launch();
}

void launch_mixed_step(const SemGeom& g, const SemBasis& b, const SemClassTables<double>& tab, const ApplyConfig* op,
                       const double* rhs, double* x, double* q, double* r, float* x32, float* r32, float* p32,
                       float* q32, const prec_t<float>* P32, double* partials, MixedCtl* ctl, PcgState* st32,
                       PcgState* gate, cudaStream_t s) {
  const long long nb = g.nb;
  k_mixed_gate<<<1, 32, 0, s>>>(ctl, st32, gate);
  k_mixed_fold<<<sem_vec_blocks(), kVecThreads, 0, s>>>(nb, x, x32, p32, q, ctl, st32);
  // mixed solves are reproducible to rounding only (FP32 atomic adds in the
  // inner operator): the refinement's FP64 operator takes atomic edge and
  // vertex adds too, not the fixed-order sums' extra pass
  ApplyConfig op_atomic = op != nullptr ? *op : ApplyConfig{};
  op_atomic.ev = nullptr;
  launch_tpt_apply<double>(g, b, tab, x, q, partials, gate, s, &op_atomic);
  k_mixed_residual<<<sem_vec_blocks(), kVecThreads, 0, s>>>(nb, rhs, q, r, partials, ctl, st32);
  k_mixed_rebase<<<sem_vec_blocks(), kVecThreads, 0, s>>>(nb, r, P32, r32, partials, ctl, st32);
  k_mixed_dir<<<sem_vec_blocks(), kVecThreads, 0, s>>>(nb, r32, p32, q32, P32, ctl, st32);
  sem_count_launch(5);
}

template <typename T>
void launch_pcg_update(long long nb, T* r, const T* q, const prec_t<T>* P, double* partials, PcgState* st,
                       cudaStream_t s) {
  k_pcg_update<T><<<num_sms() * 2, kVecThreads, 0, s>>>(nb, r, q, P, partials, st);
  sem_count_launch();
}

template <typename T>
void launch_pcg_dir(long long nb, T* x, const T* r, T* p, T* q, const prec_t<T>* P, PcgState* st, cudaStream_t s) {
  k_pcg_dir<T><<<num_sms() * 2, kVecThreads, 0, s>>>(nb, x, r, p, q, P, st);
  sem_count_launch();
}

// Shared memory of the one-pass step for a vector of nb values: z of
// ceil(nv / SMs) packs per CTA; the step is taken only up to kStepSmemMax.
// (Where z does not fit, forming it again after the barrier from r and P
// was measured slower than the two-kernel step, whose re-reads hit L2.)
constexpr size_t kStepSmemMax = 200 * 1024;
template <typename T>
static size_t step_smem(long long nb) {
  const long long nv = nb / (16 / (long long)sizeof(T));
  const long long per = (nv + num_sms() - 1) / num_sms();
  return (size_t)(per > 0 ? per : 1) * 16;
}

template <typename T>
cudaError_t prepare_pcg_step(long long nb, bool* usable) {
  *usable = false;
  cudaError_t e = cudaFuncSetAttribute(k_pcg_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStepSmemMax);
  if (e != cudaSuccess) return e;
  int dev = 0, coop = 0, occ = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  const size_t smem = step_smem<T>(nb);
  if (smem > kStepSmemMax) return cudaSuccess;   // z does not fit: two kernels
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg_step<T>, kStepThreads, smem);
  if (e != cudaSuccess) return e;
  *usable = coop != 0 && occ >= 1;
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_pcg_step(long long nb, T* x, T* r, T* p, T* q, const prec_t<T>* P, double* partials, PcgState* st,
                            cudaStream_t s) {
  const size_t smem = step_smem<T>(nb);
  if (smem > kStepSmemMax) return cudaErrorInvalidValue;   // prepare_pcg_step reports it unusable
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)num_sms());
  cfg.blockDim = dim3(kStepThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_pcg_step<T>, nb, x, r, p, q, P, partials, st);
  sem_count_launch();
  return e;
}

template <typename T>
void launch_pcg_flush(long long nb, T* x, const T* p, PcgState* st, cudaStream_t s) {
  k_pcg_flush<T><<<sem_vec_blocks(), kVecThreads, 0, s>>>(nb, x, p, st);
  sem_count_launch();
}

#define SEM_INST_VEC(T)                                                                                       \
  template void launch_pcg_init<T>(long long, const T*, T*, T*, T*, T*, const prec_t<T>*, double*, PcgState*,  \
                                   double, int, int, cudaStream_t);                                           \
  template void launch_pcg_update<T>(long long, T*, const T*, const prec_t<T>*, double*, PcgState*,           \
                                     cudaStream_t);                                                           \
  template void launch_pcg_dir<T>(long long, T*, const T*, T*, T*, const prec_t<T>*, PcgState*, cudaStream_t); \
  template void launch_pcg_flush<T>(long long, T*, const T*, PcgState*, cudaStream_t);                     \
  template cudaError_t prepare_pcg_step<T>(long long, bool*);                                                 \
  template cudaError_t launch_pcg_step<T>(long long, T*, T*, T*, T*, const prec_t<T>*, double*, PcgState*,     \
                                          cudaStream_t);
SEM_INST_VEC(double)
SEM_INST_VEC(float)

void launch_ir_residual(long long nb, const double* b, const double* Ax, double* r, double* partials,
                        PcgState* st, cudaStream_t s) {
  k_ir_residual<<<sem_vec_blocks(), kVecThreads, 0, s>>>(nb, b, Ax, r, partials, st);
  sem_count_launch();
}

void launch_scale_to_f32(long long n, const double* in, double scale, float* out, cudaStream_t s) {
  k_scale_to_f32<<<grid_for(n, 256), 256, 0, s>>>(n, in, scale, out);
  sem_count_launch();
}

void launch_ir_update(long long nb, double* x, const float* c, double scale, cudaStream_t s) {
  k_ir_update<<<grid_for(nb, 256), 256, 0, s>>>(nb, x, c, scale);
  sem_count_launch();
}

// ---------------------------------------------------------------------------
// Adjoint (differentiable solve) support
// ---------------------------------------------------------------------------
namespace {

// out = g / m at free nodes (m the assembled lumped mass), 0 on the boundary.
__global__ void k_mass_divide(SemGeom g, const double* __restrict__ mxs, const double* __restrict__ mys,
                              const double* __restrict__ mzs, const double* __restrict__ in, double* __restrict__ out,
                              int multiply) {
  const long long N = g.Nx * g.Ny * g.Nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
    const long long gx = t % g.Nx, r = t / g.Nx, gy = r % g.Ny, gz = r / g.Ny;
    const bool bnd = gx == 0 || gx == g.Nx - 1 || gy == 0 || gy == g.Ny - 1 || gz == 0 || gz == g.Nz - 1;
    const double m = mxs[gx] * mys[gy] * mzs[gz];
    out[t] = bnd ? 0.0 : (multiply ? in[t] * m : in[t] / m);
  }
}

// Per element: E[0] = w^T (M(x)M(x)M) u, E[1] = w^T (M(x)M(x)K) u, E[2] = w^T (M(x)K(x)M) u,
// E[3] = w^T (K(x)M(x)M) u on the reference element (metric factors excluded),
// E[4] = sum w_a w_b w_c w(node) f(node).  One CTA per element, local arrays
// in shared memory, each 1D stiffness product done line by line.
__global__ void k_element_forms(SemGeom g, const double* __restrict__ wgll, const double* __restrict__ Kmat,
                                const double* __restrict__ wf, const double* __restrict__ uf,
                                const double* __restrict__ ff, double* __restrict__ E) {
  extern __shared__ double sh[];
  const int p = g.p, q = p + 1, q3 = q * q * q;
  double* sw = sh;
  double* su = sh + q3;
  double* sK = su + q3;
  double* sg = sK + q * q;
  double* red = sg + q;   // [5][32]
  for (int t = threadIdx.x; t < q * q; t += blockDim.x) sK[t] = Kmat[t];
  for (int t = threadIdx.x; t < q; t += blockDim.x) sg[t] = wgll[t];
  for (long long e = blockIdx.x; e < g.nelem; e += gridDim.x) {
    int ex, ey, ez;
    semdev::elem_coords(g, e, &ex, &ey, &ez);
    __syncthreads();
    double acc[5] = {0, 0, 0, 0, 0};
    for (int t = threadIdx.x; t < q3; t += blockDim.x) {
      const int a = t % q, b = (t / q) % q, c = t / (q * q);
      const long long gi = (long long)ex * p + a + g.Nx * ((long long)ey * p + b + g.Ny * ((long long)ez * p + c));
      sw[t] = wf[gi];
      su[t] = uf[gi];
      acc[4] += sg[a] * sg[b] * sg[c] * wf[gi] * ff[gi];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < q3; t += blockDim.x) {
      const int a = t % q, b = (t / q) % q, c = t / (q * q);
      const double wv = sw[t];
      double kx = 0.0, ky = 0.0, kz = 0.0;
      for (int m = 0; m < q; ++m) {
        kx = fma(sK[a * q + m], su[(c * q + b) * q + m], kx);
        ky = fma(sK[b * q + m], su[(c * q + m) * q + a], ky);
        kz = fma(sK[c * q + m], su[(m * q + b) * q + a], kz);
      }
      acc[0] += sg[a] * sg[b] * sg[c] * wv * su[t];
      acc[1] += sg[b] * sg[c] * wv * kx;
      acc[2] += sg[a] * sg[c] * wv * ky;
      acc[3] += sg[a] * sg[b] * wv * kz;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      double x = acc[k];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) red[k * 32 + wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
      double s = 0.0;
      for (int i = 0; i < nw; ++i) s += red[threadIdx.x * 32 + i];
      E[e * 5 + threadIdx.x] = s;
    }
  }
}

// dJ/dh for one axis: for each width index i, sum over the elements in that
// slab of -(dd/dh) . E[0..3] + (dJ_e/dh) E[4], with d = J (lambda, 4/h1^2,
// 4/h2^2, 4/h3^2) and J = h1 h2 h3 / 8.  axis 0: h1 = hx[ex], etc.
__global__ void k_width_gradient(SemGeom g, int axis, const double* __restrict__ hx, const double* __restrict__ hy,
                                 const double* __restrict__ hz, double lambda, const double* __restrict__ E,
                                 double* __restrict__ out) {
  const int m = axis == 0 ? g.mx : (axis == 1 ? g.my : g.mz);
  for (int i = blockIdx.x; i < m; i += gridDim.x) {
    const long long cnt = g.nelem / m;
    double s = 0.0;
    for (long long t = threadIdx.x; t < cnt; t += blockDim.x) {
      long long ex, ey, ez;
      if (axis == 0) { ex = i; ey = t % g.my; ez = t / g.my; }
      else if (axis == 1) { ey = i; ex = t % g.mx; ez = t / g.mx; }
      else { ez = i; ex = t % g.mx; ey = t / g.mx; }
      const long long e = ex + g.mx * (ey + (long long)g.my * ez);
      const double h[3] = {hx[ex], hy[ey], hz[ez]};
      const double ha = h[axis], hb = h[(axis + 1) % 3], hc = h[(axis + 2) % 3];
      const double J = h[0] * h[1] * h[2] / 8.0, dJ = hb * hc / 8.0;   // dJ/dh_axis
      // d_k = J * 4 / h_k^2 for k = 1..3 (k - 1 = axis of that width)
      double dd[4];
      dd[0] = lambda * dJ;
      for (int k = 0; k < 3; ++k) {
        const double hk = h[k];
        dd[k + 1] = (k == axis) ? (4.0 * dJ / (hk * hk) - 8.0 * J / (hk * hk * hk)) : 4.0 * dJ / (hk * hk);
      }
      (void)ha;
      const double* Ee = E + e * 5;
      s += -(dd[0] * Ee[0] + dd[1] * Ee[1] + dd[2] * Ee[2] + dd[3] * Ee[3]) + dJ * Ee[4];
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int k = 0; k < (int)((blockDim.x + 31) >> 5); ++k) tot += red[k];
      out[i] = tot;
    }
    __syncthreads();
  }
}

// dJ/dlambda = -sum_free w m u and the same pass' partial sums (deterministic).
__global__ void k_lambda_gradient(SemGeom g, const double* __restrict__ mxs, const double* __restrict__ mys,
                                  const double* __restrict__ mzs, const double* __restrict__ w,
                                  const double* __restrict__ u, double* __restrict__ partials, double* __restrict__ out,
                                  unsigned int* counter) {
  const long long N = g.Nx * g.Ny * g.Nz;
  double s = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
    const long long gx = t % g.Nx, r = t / g.Nx, gy = r % g.Ny, gz = r / g.Ny;
    const bool bnd = gx == 0 || gx == g.Nx - 1 || gy == 0 || gy == g.Ny - 1 || gz == 0 || gz == g.Nz - 1;
    if (!bnd) s = fma(w[t] * mxs[gx] * mys[gy] * mzs[gz], u[t], s);
  }
  double v[1] = {s}, tot[1];
  if (semdev::reduce_grid<1>(v, partials, counter, tot) && threadIdx.x == 0) *out = -tot[0];
}

}  // namespace

void launch_mass_divide(const SemGeom& g, const double* mxs, const double* mys, const double* mzs, const double* in,
                        double* out, int multiply, cudaStream_t s) {
  k_mass_divide<<<grid_for(g.Nx * g.Ny * g.Nz, 256), 256, 0, s>>>(g, mxs, mys, mzs, in, out, multiply);
  sem_count_launch();
}

void launch_element_forms(const SemGeom& g, const double* wgll, const double* K, const double* w, const double* u,
                          const double* f, double* E, cudaStream_t s) {
  const int q = g.p + 1;
  const size_t smem = (size_t)(2 * q * q * q + q * q + q + 5 * 32) * sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_element_forms, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  k_element_forms<<<grid_for(g.nelem, 1, 8), 256, smem, s>>>(g, wgll, K, w, u, f, E);
  sem_count_launch();
}

void launch_width_gradient(const SemGeom& g, int axis, const double* hx, const double* hy, const double* hz,
                           double lambda, const double* E, double* out, cudaStream_t s) {
  const int m = axis == 0 ? g.mx : (axis == 1 ? g.my : g.mz);
  k_width_gradient<<<m < 4096 ? m : 4096, 256, 0, s>>>(g, axis, hx, hy, hz, lambda, E, out);
  sem_count_launch();
}

void launch_lambda_gradient(const SemGeom& g, const double* mxs, const double* mys, const double* mzs,
                            const double* w, const double* u, double* partials, double* out, unsigned int* counter,
                            cudaStream_t s) {
  k_lambda_gradient<<<sem_vec_blocks(), kVecThreads, 0, s>>>(g, mxs, mys, mzs, w, u, partials, out, counter);
  sem_count_launch();
}

SEM_DEBUG_TU(kernels)
