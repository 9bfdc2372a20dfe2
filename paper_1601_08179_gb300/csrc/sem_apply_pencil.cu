// Pencil variant of the transformed condensed operator (Sec. 6 of the paper),
// FP32, 5 <= n <= 8: the inner operator of the mixed-precision solve.
//
// The element operator is the one of the other kernels: expansion of the six
// faces into the interior eigenspace (Table 2), -D^-1, contraction back onto
// the faces, plus the primary part H~_BB restricted to the skeleton, with the
// class coefficient blocks of plane_layout(n).  Only the mapping differs.
//
// * A 256-thread CTA holds E = 256 / n^2 elements per round in shared memory
//   (faces, edges, vertices, class block, and the n^3 cube of D^-1 x).
// * Pass 1: one thread per x-pencil (j, k) of an element (n^2 per element)
//   forms the n points of the pencil (six face terms each), scales them by
//   D^-1 (one reciprocal per point), writes them to the cube and contracts
//   them over i in its registers: the two x-face outputs at (k, j) are
//   complete there.
// * Pass 2: one thread per (i, m) reads two columns of the cube, along j at
//   k = m (the y-face outputs at (k, i)) and along k at j = m (the z-face
//   outputs at (j, i)); the same threads then form the edge and vertex
//   outputs (primary part only: edges and vertices do not couple to the
//   interior) from line sums of the gathered faces.
// * No shuffles and no lane selections: the three contractions are a register
//   sum and two strided column sums.  Every output is scatter-added
//   (red.global.add) and the element share of x^T (A x) accumulated.
// * Elements are visited x fastest, a round takes E consecutive ones (their
//   x-faces are adjacent in the face array), CTAs take contiguous ranges.

#include <cuda_runtime.h>

#include "sem_device.cuh"
#include "sem_kernels.cuh"

using namespace semdev;

namespace {

constexpr int kPencilThreads = 256;
constexpr int kPencilHdr = 32;   // ints per element: 26 entity offsets, class

template <int N>
struct PencilSm {
  static constexpr int RS = 8;                  // padded row (rows of faces and of the cube)
  static constexpr int FS = N * RS;
  static constexpr int E = kPencilThreads / (N * N);   // elements per round
  static constexpr int F = 0;                   // faces [6][N][RS]
  static constexpr int EX = 6 * FS;             // x-edges [4][RS] (sb + 2 sc), y-edges [4][RS] (4 + sa + 2 sc)
  static constexpr int EZ = EX + 8 * RS;        // z-edges [N][4] (component sa + 2 sb)
  static constexpr int VT = EZ + 4 * N;         // vertices [8]
  static constexpr int C = VT + 8;              // class block (plane_layout(N), rs = 8)
  static constexpr int PCS = 5 * RS + 4 * N + 36;
  static constexpr int CUBE = (C + PCS + 3) & ~3;   // D^-1 x, [k][j][RS]
  static constexpr int size = CUBE + N * N * RS + 4;  // + 4: slots start 4 banks apart
  static_assert(EX % 4 == 0 && EZ % 4 == 0 && VT % 4 == 0 && C % 4 == 0 && CUBE % 4 == 0 && size % 4 == 0 &&
                    PCS % 4 == 0,
                "16-byte alignment");
  static_assert(E >= 1 && E * N * N <= kPencilThreads, "a thread per pencil");
};

template <int M>
__device__ __forceinline__ void pload(const float* p, float (&r)[M]) {
#pragma unroll
  for (int t = 0; t < M; t += 4) {
    const float4 v = *reinterpret_cast<const float4*>(p + t);
    r[t] = v.x;
    r[t + 1] = v.y;
    r[t + 2] = v.z;
    r[t + 3] = v.w;
  }
}

// Entity offsets (-1: Dirichlet or no element) and class of the round's
// elements e0 .. e0 + E - 1 into their headers.
template <int N>
__device__ __forceinline__ void pencil_headers(const SemGeom& g, const SemClassTables<float>& tab,
                                               const EntityAffine* ent, long long e0, int* hdr) {
  using S = PencilSm<N>;
  for (int t = threadIdx.x; t < S::E * 27; t += kPencilThreads) {
    const int el = t / 27, r = t - el * 27;
    const long long e = e0 + el;
    const bool live = e < g.nelem;
    int ex = 0, ey = 0, ez = 0;
    if (live) {
      const int mxy = g.mx * g.my;
      ez = (int)(e / mxy);
      const int rem = (int)(e - (long long)ez * mxy);
      ey = rem / g.mx;
      ex = rem - ey * g.mx;
    }
    int val;
    if (r == 26) {
      val = live ? elem_class(g, tab, ex, ey, ez) : 0;
    } else {
      const int bits = (ex == 0) | ((ex == g.mx - 1) << 1) | ((ey == 0) << 2) | ((ey == g.my - 1) << 3) |
                       ((ez == 0) << 4) | ((ez == g.mz - 1) << 5);
      val = live ? entity_offset(ent[r], r, bits, ex, ey, ez, g) : -1;
    }
    hdr[el * kPencilHdr + r] = val;
  }
}

// Gather R^T of the round's elements (zero fill on Dirichlet entities) and
// their class blocks, as cp.async copies.
template <int N>
__device__ __forceinline__ void pencil_gather(const SemClassTables<float>& tab, const float* __restrict__ u,
                                              const int* hdr, float* slots) {
  using S = PencilSm<N>;
  constexpr int NF = 6 * N * N, NE = 12 * N, PER = NF + NE + 8;
  for (int t = threadIdx.x; t < S::E * PER; t += kPencilThreads) {
    const int el = t / PER, r = t - el * PER;
    const int* H = hdr + el * kPencilHdr;
    float* W = slots + el * S::size;
    int off, idx;
    float* dst;
    if (r < NF) {
      const int slot = r / (N * N), q = r - slot * N * N, row = q / N, col = q - row * N;
      off = H[slot];
      idx = q;
      dst = W + S::F + slot * S::FS + row * S::RS + col;
    } else if (r < NF + NE) {
      const int q = r - NF, slot = q / N, l = q - slot * N;
      off = H[6 + slot];
      idx = l;
      dst = slot < 8 ? W + S::EX + slot * S::RS + l : W + S::EZ + 4 * l + (slot - 8);
    } else {
      const int v = r - NF - NE;
      off = H[18 + v];
      idx = 0;
      dst = W + S::VT + v;
    }
    cp_async4(dst, u + (off >= 0 ? off + idx : 0), off >= 0);
  }
  for (int t = threadIdx.x; t < S::E * (S::PCS / 4); t += kPencilThreads) {
    const int el = t / (S::PCS / 4), r = 4 * (t - el * (S::PCS / 4));
    cp_async16(slots + el * S::size + S::C + r, tab.plane + (long long)hdr[el * kPencilHdr + 26] * tab.plane_stride + r);
  }
}

// Pass 1: x-pencil (j, k) of element el: expansion, D^-1, the cube row, the
// x-contraction and the two x-face outputs.
template <int N>
__device__ __forceinline__ void pencil_x(float* W, const int* H, int j, int k, float* __restrict__ v, float& dot) {
  using S = PencilSm<N>;
  constexpr int RS = S::RS, FS = S::FS;
  const PlaneLayout L = plane_layout(N);
  const float* Cf = W + S::C;
  const float A = W[S::F + k * RS + j], B = W[S::F + FS + k * RS + j];
  float a[RS], b[RS], l1[RS], cr[RS], dr[RS], e4[RS], e5[RS];
  pload<RS>(Cf + L.pa, a);
  pload<RS>(Cf + L.pb, b);
  pload<RS>(Cf + L.pl1, l1);
  pload<RS>(W + S::F + 2 * FS + k * RS, cr);
  pload<RS>(W + S::F + 3 * FS + k * RS, dr);
  pload<RS>(W + S::F + 4 * FS + j * RS, e4);
  pload<RS>(W + S::F + 5 * FS + j * RS, e5);
  const float4 qj = *reinterpret_cast<const float4*>(Cf + L.pq + 4 * j);
  const float4 qk = *reinterpret_cast<const float4*>(Cf + L.pq + 4 * k);
  const float cj = qj.x, dj = qj.y, ek = qk.z, gk = qk.w;
  const float w0 = Cf[L.ps + 32], d0 = Cf[L.ps + 34];
  const float l2j = Cf[L.pl2 + j], l3k = Cf[L.pl3 + k];
  const float sjk = d0 + l2j + l3k;
  float X0 = 0.f, X1 = 0.f, wr[RS];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float x = a[i] * A;
    x = fmaf(b[i], B, x);
    x = fmaf(cj, cr[i], x);
    x = fmaf(dj, dr[i], x);
    x = fmaf(ek, e4[i], x);
    x = fmaf(gk, e5[i], x);
    const float w = x * rcp_approx(sjk + l1[i]);   // D^-1 x (the sign is applied at the outputs)
    X0 = fmaf(a[i], w, X0);
    X1 = fmaf(b[i], w, X1);
    wr[i] = w;
  }
#pragma unroll
  for (int i = N; i < RS; ++i) wr[i] = 0.f;
  float* dst = W + S::CUBE + (k * N + j) * RS;
#pragma unroll
  for (int t = 0; t < RS; t += 4) *reinterpret_cast<float4*>(dst + t) = make_float4(wr[t], wr[t + 1], wr[t + 2], wr[t + 3]);
  // x-faces at (k, j): diagonal, opposite face, the four edge lines, -condensed
  const float4 ezk = *reinterpret_cast<const float4*>(W + S::EZ + 4 * k);   // Ez[sa + 2 sb][k]
  const float ey0 = W[S::EX + 4 * RS + j], ey1 = W[S::EX + 5 * RS + j];
  const float ey2 = W[S::EX + 6 * RS + j], ey3 = W[S::EX + 7 * RS + j];
  const float bx = w0 * (l2j + l3k);
  const int kj = k * N + j;
  const int ox0 = H[0], ox1 = H[1];
  float o = (Cf[L.ps + 6] + bx) * A;
  o = fmaf(Cf[L.ps + 0], B, o);
  o = fmaf(w0, fmaf(cj, ezk.x, fmaf(dj, ezk.z, fmaf(ek, ey0, gk * ey2))), o);
  o -= X0;
  if (ox0 >= 0) {
    atomicAdd(v + ox0 + kj, o);
    dot = fmaf(A, o, dot);
  }
  o = (Cf[L.ps + 7] + bx) * B;
  o = fmaf(Cf[L.ps + 1], A, o);
  o = fmaf(w0, fmaf(cj, ezk.y, fmaf(dj, ezk.w, fmaf(ek, ey1, gk * ey3))), o);
  o -= X1;
  if (ox1 >= 0) {
    atomicAdd(v + ox1 + kj, o);
    dot = fmaf(B, o, dot);
  }
}

// Pass 2a: column i of the cube along j at k = m (y-faces at (k, i)) and
// along k at j = m (z-faces at (j, i)).
template <int N>
__device__ __forceinline__ void pencil_yz(float* W, const int* H, int m, int i, float* __restrict__ v, float& dot) {
  using S = PencilSm<N>;
  constexpr int RS = S::RS, FS = S::FS;
  const PlaneLayout L = plane_layout(N);
  const float* Cf = W + S::C;
  const float* cube = W + S::CUBE;
  const float w0 = Cf[L.ps + 32];
  const float ai = Cf[L.pa + i], bi = Cf[L.pb + i], l1i = Cf[L.pl1 + i];
  float Y0 = 0.f, Y1 = 0.f, Z4 = 0.f, Z5 = 0.f;
#pragma unroll
  for (int t = 0; t < N; ++t) {
    const float4 q = *reinterpret_cast<const float4*>(Cf + L.pq + 4 * t);   // (c, d, e, g)_t
    const float wy = cube[(m * N + t) * RS + i];    // k = m, j = t
    const float wz = cube[(t * N + m) * RS + i];    // k = t, j = m
    Y0 = fmaf(q.x, wy, Y0);
    Y1 = fmaf(q.y, wy, Y1);
    Z4 = fmaf(q.z, wz, Z4);
    Z5 = fmaf(q.w, wz, Z5);
  }
  // y-faces at (k = m, i)
  {
    const int k = m;
    const float4 qk = *reinterpret_cast<const float4*>(Cf + L.pq + 4 * k);
    const float ek = qk.z, gk = qk.w;
    const float4 ezk = *reinterpret_cast<const float4*>(W + S::EZ + 4 * k);
    const float ex0 = W[S::EX + i], ex1 = W[S::EX + RS + i], ex2 = W[S::EX + 2 * RS + i], ex3 = W[S::EX + 3 * RS + i];
    const float Cl = W[S::F + 2 * FS + k * RS + i], Dl = W[S::F + 3 * FS + k * RS + i];
    const float by = w0 * (l1i + Cf[L.pl3 + k]);
    const int ki = k * N + i;
    const int oy0 = H[2], oy1 = H[3];
    float o = (Cf[L.ps + 8] + by) * Cl;
    o = fmaf(Cf[L.ps + 2], Dl, o);
    o = fmaf(w0, fmaf(ai, ezk.x, fmaf(bi, ezk.y, fmaf(ek, ex0, gk * ex2))), o);
    o -= Y0;
    if (oy0 >= 0) {
      atomicAdd(v + oy0 + ki, o);
      dot = fmaf(Cl, o, dot);
    }
    o = (Cf[L.ps + 9] + by) * Dl;
    o = fmaf(Cf[L.ps + 3], Cl, o);
    o = fmaf(w0, fmaf(ai, ezk.z, fmaf(bi, ezk.w, fmaf(ek, ex1, gk * ex3))), o);
    o -= Y1;
    if (oy1 >= 0) {
      atomicAdd(v + oy1 + ki, o);
      dot = fmaf(Dl, o, dot);
    }
  }
  // z-faces at (j = m, i)
  {
    const int j = m;
    const float4 qj = *reinterpret_cast<const float4*>(Cf + L.pq + 4 * j);
    const float cj = qj.x, dj = qj.y;
    const float bz = w0 * (l1i + Cf[L.pl2 + j]);
    const float f4 = W[S::F + 4 * FS + j * RS + i], f5 = W[S::F + 5 * FS + j * RS + i];
    const int ji = j * N + i;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const float own = s ? f5 : f4, opp = s ? f4 : f5;
      const float xa = W[S::EX + (2 * s) * RS + i], xb = W[S::EX + (2 * s + 1) * RS + i];   // Ex[0][s], Ex[1][s]
      const float ya = W[S::EX + (4 + 2 * s) * RS + j], yb = W[S::EX + (5 + 2 * s) * RS + j];   // Ey[0][s], Ey[1][s]
      float o = (Cf[L.ps + 10 + s] + bz) * own;
      o = fmaf(Cf[L.ps + 4 + s], opp, o);
      o = fmaf(w0, fmaf(ai, ya, fmaf(bi, yb, fmaf(cj, xa, dj * xb))), o);
      o -= s ? Z5 : Z4;
      const int oz = H[4 + s];
      if (oz >= 0) {
        atomicAdd(v + oz + ji, o);
        dot = fmaf(own, o, dot);
      }
    }
  }
}

// Pass 2b: one edge point (item < 12 N: edge slot item / N at position
// item % N) or one vertex (item - 12 N), primary part only.
template <int N>
__device__ __forceinline__ void pencil_ev(float* W, const int* H, int item, float* __restrict__ v, float& dot) {
  using S = PencilSm<N>;
  constexpr int RS = S::RS, FS = S::FS;
  const PlaneLayout L = plane_layout(N);
  const float* Cf = W + S::C;
  const float* Fp = W + S::F;
  const float w0 = Cf[L.ps + 32], w02 = Cf[L.ps + 33], d0 = Cf[L.ps + 34];
  const float* V = W + S::VT;
  if (item < 12 * N) {
    const int slot = item / N, l = item - slot * N, grp = slot >> 2, q = slot & 3;
    float o, in;
    if (grp == 0) {   // x-edge Ex[sb][sc] at i = l
      const int sb = q & 1, sc = q >> 1;
      const float* ex = W + S::EX;   // ex[q'] at ex + q' RS
      float szc = 0.f, sy = 0.f;     // sum_m (c|d)_m F_{4+sc}[m][l], sum_k (e|g)_k F_{2+sb}[k][l]
#pragma unroll
      for (int t = 0; t < N; ++t) {
        const float4 c = *reinterpret_cast<const float4*>(Cf + L.pq + 4 * t);
        szc = fmaf(sb ? c.y : c.x, Fp[(4 + sc) * FS + t * RS + l], szc);
        sy = fmaf(sc ? c.w : c.z, Fp[(2 + sb) * FS + t * RS + l], sy);
      }
      in = ex[q * RS + l];
      o = (w02 * (d0 + Cf[L.pl1 + l]) + Cf[L.ps + 12 + q]) * in;
      o = fmaf(w02, fmaf(Cf[L.pa + l], V[2 * sb + 4 * sc], Cf[L.pb + l] * V[1 + 2 * sb + 4 * sc]), o);
      o = fmaf(w0, szc + sy, o);
      o = fmaf(w0 * Cf[L.ps + 2 + sb], ex[((1 - sb) + 2 * sc) * RS + l], o);
      o = fmaf(w0 * Cf[L.ps + 4 + sc], ex[(sb + 2 * (1 - sc)) * RS + l], o);
    } else if (grp == 1) {   // y-edge Ey[sa][sc] at j = l
      const int sa = q & 1, sc = q >> 1;
      const float* ey = W + S::EX + 4 * RS;
      float szr = 0.f, sx = 0.f;     // sum_m (a|b)_m F_{4+sc}[l][m], sum_k (e|g)_k F_sa[k][l]
      const float* ab = Cf + (sa ? L.pb : L.pa);
#pragma unroll
      for (int t = 0; t < N; ++t) {
        const float4 c = *reinterpret_cast<const float4*>(Cf + L.pq + 4 * t);
        szr = fmaf(ab[t], Fp[(4 + sc) * FS + l * RS + t], szr);
        sx = fmaf(sc ? c.w : c.z, Fp[sa * FS + t * RS + l], sx);
      }
      const float4 cl = *reinterpret_cast<const float4*>(Cf + L.pq + 4 * l);
      in = ey[q * RS + l];
      o = (w02 * (d0 + Cf[L.pl2 + l]) + Cf[L.ps + 16 + q]) * in;
      o = fmaf(w02, fmaf(cl.x, V[sa + 4 * sc], cl.y * V[sa + 2 + 4 * sc]), o);
      o = fmaf(w0, szr + sx, o);
      o = fmaf(w0 * Cf[L.ps + sa], ey[((1 - sa) + 2 * sc) * RS + l], o);
      o = fmaf(w0 * Cf[L.ps + 4 + sc], ey[(sa + 2 * (1 - sc)) * RS + l], o);
    } else {   // z-edge Ez[sa][sb] at k = l
      const int sa = q & 1, sb = q >> 1;
      const float* ezl = W + S::EZ + 4 * l;
      float syr = 0.f, sxr = 0.f;    // sum_m (a|b)_m F_{2+sb}[l][m], sum_m (c|d)_m F_sa[l][m]
      const float* ab = Cf + (sa ? L.pb : L.pa);
#pragma unroll
      for (int t = 0; t < N; ++t) {
        const float4 c = *reinterpret_cast<const float4*>(Cf + L.pq + 4 * t);
        syr = fmaf(ab[t], Fp[(2 + sb) * FS + l * RS + t], syr);
        sxr = fmaf(sb ? c.y : c.x, Fp[sa * FS + l * RS + t], sxr);
      }
      const float4 cl = *reinterpret_cast<const float4*>(Cf + L.pq + 4 * l);
      in = ezl[q];
      o = (w02 * (d0 + Cf[L.pl3 + l]) + Cf[L.ps + 20 + q]) * in;
      o = fmaf(w02, fmaf(cl.z, V[sa + 2 * sb], cl.w * V[sa + 2 * sb + 4]), o);
      o = fmaf(w0, syr + sxr, o);
      o = fmaf(w0 * Cf[L.ps + sa], ezl[(1 - sa) + 2 * sb], o);
      o = fmaf(w0 * Cf[L.ps + 2 + sb], ezl[sa + 2 * (1 - sb)], o);
    }
    const int off = H[6 + slot];
    if (off >= 0) {
      atomicAdd(v + off + l, o);
      dot = fmaf(in, o, dot);
    }
  } else {
    const int r = item - 12 * N, sa = r & 1, sb = (r >> 1) & 1, sc = r >> 2;
    const float* exr = W + S::EX + (sb + 2 * sc) * RS;
    const float* eyr = W + S::EX + (4 + sa + 2 * sc) * RS;
    const float* ab = Cf + (sa ? L.pb : L.pa);
    float sv = 0.f;
#pragma unroll
    for (int t = 0; t < N; ++t) {
      const float4 c = *reinterpret_cast<const float4*>(Cf + L.pq + 4 * t);
      sv = fmaf(ab[t], exr[t], sv);
      sv = fmaf(sb ? c.y : c.x, eyr[t], sv);
      sv = fmaf(sc ? c.w : c.z, W[S::EZ + 4 * t + sa + 2 * sb], sv);
    }
    const float vr = V[r];
    float o = Cf[L.ps + 24 + r] * vr;
    o = fmaf(w02, sv, o);
    o = fmaf(w02 * Cf[L.ps + sa], V[r ^ 1], o);
    o = fmaf(w02 * Cf[L.ps + 2 + sb], V[r ^ 2], o);
    o = fmaf(w02 * Cf[L.ps + 4 + sc], V[r ^ 4], o);
    const int off = H[18 + r];
    if (off >= 0) {
      atomicAdd(v + off, o);
      dot = fmaf(vr, o, dot);
    }
  }
}

template <int N>
__global__ void __launch_bounds__(kPencilThreads, 3)
k_tpt_apply_pencil(SemGeom g, SemClassTables<float> tab, const float* __restrict__ u, float* __restrict__ v,
                   double* __restrict__ partials, PcgState* st) {
  using S = PencilSm<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ EntityAffine ent[26];
  if (st != nullptr && st->done) return;
  if (threadIdx.x < 26) entity_affine(g, threadIdx.x, &ent[threadIdx.x]);
  int* hdr = reinterpret_cast<int*>(smem_raw);
  float* slots = reinterpret_cast<float*>(smem_raw + (size_t)S::E * kPencilHdr * sizeof(int));
  // rounds of E consecutive elements, split into equal contiguous ranges over the grid
  const long long nr = (g.nelem + S::E - 1) / S::E;
  const long long r_begin = nr * blockIdx.x / gridDim.x, r_end = nr * (blockIdx.x + 1) / gridDim.x;
  const int tid = threadIdx.x;
  float dot = 0.f;
  for (long long rd = r_begin; rd < r_end; ++rd) {
    __syncthreads();   // the previous round is done with the slots (and ent is ready)
    pencil_headers<N>(g, tab, ent, rd * S::E, hdr);
    __syncthreads();
    pencil_gather<N>(tab, u, hdr, slots);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    if (tid < S::E * N * N) {
      const int el = tid / (N * N), r = tid - el * N * N, k = r / N, j = r - k * N;
      pencil_x<N>(slots + el * S::size, hdr + el * kPencilHdr, j, k, v, dot);
    }
    __syncthreads();
    if (tid < S::E * N * N) {
      const int el = tid / (N * N), r = tid - el * N * N, m = r / N, i = r - m * N;
      pencil_yz<N>(slots + el * S::size, hdr + el * kPencilHdr, m, i, v, dot);
    }
    for (int t = tid; t < S::E * (12 * N + 8); t += kPencilThreads) {
      const int el = t / (12 * N + 8), item = t - el * (12 * N + 8);
      pencil_ev<N>(slots + el * S::size, hdr + el * kPencilHdr, item, v, dot);
    }
  }
  if (st != nullptr) {
    double vals[1] = {(double)dot}, tot[1];
    if (reduce_grid<1>(vals, partials, &st->counter[0], tot) && threadIdx.x == 0) {
      const double pq = tot[0];
      st->pq = pq;
      if (!(pq > 0.0) || !isfinite(pq)) st->done = 2;
      else st->alpha = st->rho / pq;
    }
  }
}

template <int N>
size_t pencil_smem() {
  using S = PencilSm<N>;
  return (size_t)S::E * kPencilHdr * sizeof(int) + (size_t)S::E * S::size * sizeof(float);
}

template <int N>
void launch_pencil_n(const SemGeom& g, const SemClassTables<float>& t, const float* x, float* y, double* partials,
                     PcgState* st, cudaStream_t s) {
  using S = PencilSm<N>;
  const size_t smem = pencil_smem<N>();
  static bool attr = false;
  if (!attr) {   // once per instantiation; the first launch happens outside any capture
    cudaFuncSetAttribute(k_tpt_apply_pencil<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tpt_apply_pencil<N>, kPencilThreads, smem);
  if (occ < 1) occ = 1;
  const long long rounds = (g.nelem + S::E - 1) / S::E;
  long long grid = (long long)sem_num_sms() * occ;
  if (grid > rounds) grid = rounds;
  k_tpt_apply_pencil<N><<<(int)grid, kPencilThreads, smem, s>>>(g, t, x, y, partials, st);
  sem_count_launch();
}

}  // namespace

bool pencil_supported(int n) { return n >= 5 && n <= 8; }

void launch_pencil_apply(const SemGeom& g, const SemClassTables<float>& t, const float* x, float* y,
                         double* partials, PcgState* st, cudaStream_t s) {
  switch (g.n) {
    case 5: launch_pencil_n<5>(g, t, x, y, partials, st, s); break;
    case 6: launch_pencil_n<6>(g, t, x, y, partials, st, s); break;
    case 7: launch_pencil_n<7>(g, t, x, y, partials, st, s); break;
    default: launch_pencil_n<8>(g, t, x, y, partials, st, s); break;
  }
}

SEM_DEBUG_TU(pencil)
