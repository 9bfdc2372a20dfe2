// Plane-per-lane variant of the transformed condensed operator (Sec. 6 of the
// paper), for FP32 and 2 <= n <= 8: the inner operator of the mixed-precision
// solve.
//
// The element operator is the one of the CTA-tile kernel (sem_apply.cu):
// expansion of the six faces into the interior eigenspace (Table 2), -D^-1,
// contraction back onto the faces, plus the primary part H~_BB restricted to
// the skeleton; only the mapping of the work onto the GPU differs.
//
// * A group of G = 4 (n <= 4) or 8 lanes owns one element; a warp holds
//   32 / G elements.  Lane j of a group owns the y-plane j of the n^3 cube
//   and walks it in k, i.e. it holds a row of n points at a time.
// * The x-contraction (sum over i) and the z-contraction (sum over k) are
//   done in the lane's registers; the y-contraction (sum over j) is a
//   butterfly reduce-scatter over the group (shuffles), after which lane i
//   holds the y-face outputs at (k, i).
// * D^-1 = 1 / (d0 + d1 lambda_i + d2 lambda_j + d3 lambda_k) (the diagonal
//   of H~_II in the eigenbasis) is formed with one reciprocal per point, and
//   the face, edge and vertex diagonals of H~_BB are formed from the same
//   lambda vectors, so a class's coefficient block is 9n + O(1) numbers.
// * The line sums of the primary part that run along k are accumulated in
//   the same k walk; the others are one row or column of shared memory per
//   lane, the edge position being the lane index.
// * Face rows are padded to four floats (16-byte vector loads), and the
//   element slots of a warp are offset by 32 / (elements per warp) banks, so
//   a broadcast row load of the whole warp is one shared-memory wavefront.

#include <cuda_runtime.h>

#include "sem_device.cuh"
#include "sem_kernels.cuh"

using namespace semdev;

namespace {

constexpr int kPlaneThreads = 96;
constexpr int kHdr = 32;   // ints per element slot: 26 entity offsets, class, loaded class

template <int N>
struct PlaneSm {
  static constexpr int G = N <= 4 ? 4 : 8;     // lanes per element
  static constexpr int EPW = 32 / G;           // elements per warp
  static constexpr int RS = (N + 3) & ~3;      // padded row
  static constexpr int FS = N * RS;            // padded face
  static constexpr int F = 0;                  // faces [6][N][RS]
  static constexpr int EX = 6 * FS;            // x-edges [4][RS] (slot sb + 2 sc), y-edges [4][RS] (4 + sa + 2 sc)
  static constexpr int EZ = EX + 8 * RS;       // z-edges [N][4], component sa + 2 sb
  static constexpr int VT = EZ + 4 * N;        // vertices [8]
  static constexpr int C = VT + 8;             // class coefficient block (plane_layout)
  static constexpr int PCS = 5 * RS + 4 * N + 36;
  static constexpr int raw = C + PCS;
  static constexpr int step = 32 / EPW;        // bank offset between the element slots of a warp
  static constexpr int size = raw + ((step - raw % 32) % 32 + 32) % 32;
  static_assert(size % 32 == step, "slot stride");
  static_assert(EX % 4 == 0 && EZ % 4 == 0 && VT % 4 == 0 && C % 4 == 0, "16-byte alignment");
};

// M floats from a 16-byte aligned row (M a multiple of 4).
template <int M>
__device__ __forceinline__ void load_row(const float* p, float (&r)[M]) {
#pragma unroll
  for (int t = 0; t < M; t += 4) {
    const float4 v = *reinterpret_cast<const float4*>(p + t);
    r[t] = v.x;
    r[t + 1] = v.y;
    r[t + 2] = v.z;
    r[t + 3] = v.w;
  }
}

// Sums P0[i], P1[i] over the G lanes of a group; lane jl of the group ends
// with the sums for i = jl.  Each halving step keeps the half of the index
// range named by one bit of jl and adds the partner's copy of it.
template <int H, int G>
__device__ __forceinline__ void halve(float (&P0)[G], float (&P1)[G], int jl) {
  const bool up = (jl & H) != 0;
#pragma unroll
  for (int t = 0; t < H; ++t) {
    const float s0 = up ? P0[t] : P0[t + H], k0 = up ? P0[t + H] : P0[t];
    const float s1 = up ? P1[t] : P1[t + H], k1 = up ? P1[t + H] : P1[t];
    P0[t] = k0 + __shfl_xor_sync(0xffffffffu, s0, H);
    P1[t] = k1 + __shfl_xor_sync(0xffffffffu, s1, H);
  }
}

// The first halving step of the sums of cj W[i] and dj W[i] over the lanes
// (cj, dj the lane's own factors): the selection is made on W, so each lane
// forms only the products it sends and folds its kept half in with one FMA.
template <int H, int G>
__device__ __forceinline__ void halve_w(const float (&W)[G], float cj, float dj, float (&P0)[G], float (&P1)[G],
                                        int jl) {
  const bool up = (jl & H) != 0;
#pragma unroll
  for (int t = 0; t < H; ++t) {
    const float ws = up ? W[t] : W[t + H], wk = up ? W[t + H] : W[t];
    P0[t] = fmaf(cj, wk, __shfl_xor_sync(0xffffffffu, cj * ws, H));
    P1[t] = fmaf(dj, wk, __shfl_xor_sync(0xffffffffu, dj * ws, H));
  }
}

// Sums cj W[i] and dj W[i] over the G lanes of a group; lane jl ends with the
// sums for i = jl.
template <int G>
__device__ __forceinline__ void reduce_scatter(const float (&W)[G], float cj, float dj, int jl, float* y0,
                                               float* y1) {
  float P0[G], P1[G];
  halve_w<G / 2, G>(W, cj, dj, P0, P1, jl);
  if constexpr (G == 8) halve<2, G>(P0, P1, jl);
  halve<1, G>(P0, P1, jl);
  *y0 = P0[0];
  *y1 = P1[0];
}

// Sums P[i] and sigma_j P[i] over the G lanes of a group (sigma_j = (-1)^j,
// j = lane), lane jl ending with the two sums for i = jl.  The first halving
// step pairs lanes of opposite parity and forms P_j + P_{j^1} and
// P_j - P_{j^1} (the second is the pair's signed sum up to sigma_j); the
// later steps pair lanes of equal parity, so both sums just add; the sign
// sigma_jl is applied at the end.
template <int G>
__device__ __forceinline__ void reduce_scatter_parity(const float (&P)[G], int jl, float* y0, float* y1) {
  const bool odd = (jl & 1) != 0;
  float s[G / 2], d[G / 2];   // index i = 2 t + (jl & 1)
#pragma unroll
  for (int t = 0; t < G / 2; ++t) {
    const float keep = odd ? P[2 * t + 1] : P[2 * t], send = odd ? P[2 * t] : P[2 * t + 1];
    const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
    s[t] = keep + recv;
    d[t] = keep - recv;
  }
  float S, D;
  if constexpr (G == 8) {
    const bool up = (jl & 2) != 0;
    float s2[2], d2[2];   // index i = 4 u + 2 up + (jl & 1)
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const float ks = up ? s[2 * u + 1] : s[2 * u], ss = up ? s[2 * u] : s[2 * u + 1];
      const float kd = up ? d[2 * u + 1] : d[2 * u], sd = up ? d[2 * u] : d[2 * u + 1];
      s2[u] = ks + __shfl_xor_sync(0xffffffffu, ss, 2);
      d2[u] = kd + __shfl_xor_sync(0xffffffffu, sd, 2);
    }
    const bool hi = (jl & 4) != 0;
    const float ks = hi ? s2[1] : s2[0], ss = hi ? s2[0] : s2[1];
    const float kd = hi ? d2[1] : d2[0], sd = hi ? d2[0] : d2[1];
    S = ks + __shfl_xor_sync(0xffffffffu, ss, 4);
    D = kd + __shfl_xor_sync(0xffffffffu, sd, 4);
  } else {
    const bool up = (jl & 2) != 0;
    const float ks = up ? s[1] : s[0], ss = up ? s[0] : s[1];
    const float kd = up ? d[1] : d[0], sd = up ? d[0] : d[1];
    S = ks + __shfl_xor_sync(0xffffffffu, ss, 2);
    D = kd + __shfl_xor_sync(0xffffffffu, sd, 2);
  }
  *y0 = S;
  *y1 = odd ? -D : D;
}

// Offsets of the element's 26 entities (-1: Dirichlet entity or no element)
// and its class (fallback for a missing element) into H[0..26].
template <int G>
__device__ __forceinline__ void plane_header(const SemGeom& g, const SemClassTables<float>& tab,
                                             const EntityAffine* ent, int e, bool live, int fallback, int jl,
                                             int* H) {
  int ex = 0, ey = 0, ez = 0;
  // x fastest: the element groups of a warp are neighbours in x, whose faces,
  // edges and vertices are adjacent in every entity array (measured faster
  // than visiting the graded axis slowest, which shares class blocks instead)
  if (live) { const int mxy = g.mx * g.my; ez = e / mxy; const int r = e - ez * mxy; ey = r / g.mx; ex = r - ey * g.mx; }
  const int bits = (ex == 0) | ((ex == g.mx - 1) << 1) | ((ey == 0) << 2) | ((ey == g.my - 1) << 3) |
                   ((ez == 0) << 4) | ((ez == g.mz - 1) << 5);
  for (int r = jl; r < 27; r += G) {
    int val;
    if (r == 26) {
      val = live ? elem_class(g, tab, ex, ey, ez) : fallback;
    } else {
      const EntityAffine a = ent[r];
      val = live ? entity_offset(a, r, bits, ex, ey, ez, g) : -1;
    }
    H[r] = val;
  }
}

// Issues the asynchronous gather R^T of one element (entity offsets in H)
// into the slot buffer W: faces row by row with the lane as the column,
// edges one value per lane, vertices; and the class block when load_cls.
template <int N>
__device__ __forceinline__ void plane_gather(const float* __restrict__ u, const float* cls_src, bool load_cls,
                                             const int* H, float* W, int jl) {
  using S = PlaneSm<N>;
  if (jl < N) {
#pragma unroll
    for (int slot = 0; slot < 6; ++slot) {
      const int off = H[slot];
      const float* src = u + (off >= 0 ? off : 0) + jl;
      float* dst = W + S::F + slot * S::FS + jl;
#pragma unroll
      for (int row = 0; row < N; ++row) cp_async4(dst + row * S::RS, src + row * N, off >= 0);
    }
#pragma unroll
    for (int slot = 0; slot < 12; ++slot) {
      const int off = H[6 + slot];
      float* dst = slot < 8 ? W + S::EX + slot * S::RS + jl : W + S::EZ + 4 * jl + (slot - 8);
      cp_async4(dst, u + (off >= 0 ? off : 0) + jl, off >= 0);
    }
  }
  for (int r = jl; r < 8; r += S::G) {
    const int off = H[18 + r];
    cp_async4(W + S::VT + r, u + (off >= 0 ? off : 0), off >= 0);
  }
  if (load_cls)
    for (int r = 4 * jl; r < S::PCS; r += 4 * S::G) cp_async16(W + S::C + r, cls_src + r);
}

// The element operator of one element whose gathered values sit in W
// (offsets in H); scatter-adds into v and accumulates x^T (A x) into dot.
template <int N>
__device__ __forceinline__ void plane_element(float* W, const int* H, float* __restrict__ v, int jl,
                                              float& dot) {
  using S = PlaneSm<N>;
  constexpr int G = S::G, RS = S::RS, FS = S::FS;
  constexpr int PA = 0, PB = RS, PL1 = 2 * RS, PL2 = 3 * RS, PL3 = 4 * RS, PQ = 5 * RS, PS = 5 * RS + 4 * N;
  const float* Fp = W + S::F;
  const float* Cf = W + S::C;
  const bool act = jl < N;                 // lanes past n mirror plane n-1 and contribute zeros
  const int j = act ? jl : N - 1;
    // ---- per-element constants of this lane
    const float w0 = Cf[PS + 32], w02 = Cf[PS + 33], d0 = Cf[PS + 34];
    // The 1D border vectors are centro-symmetric: K~_{Ip}[c] = (-1)^c K~_{I0}[c]
    // (the GLL points and the interior eigenproblem are symmetric under
    // x -> -x, so eigenvector c is even or odd with c; canonical signs), hence
    // b_i = (-1)^i a_i, d_j = (-1)^j c_j and g_k = (-1)^k e_k: each pair of
    // expansion terms is one term, and each pair of contractions a sum over
    // the even and one over the odd indices.
    float a[RS], l1[RS], e45p[RS], e45m[RS];   // e45p/m = z-face rows j: F4 + F5, F4 - F5
    load_row<RS>(Cf + PA, a);
    load_row<RS>(Cf + PL1, l1);
    load_row<RS>(Fp + 4 * FS + j * RS, e45p);
    load_row<RS>(Fp + 5 * FS + j * RS, e45m);
#pragma unroll
    for (int i = 0; i < RS; ++i) {
      const float f4 = e45p[i], f5 = e45m[i];
      e45p[i] = f4 + f5;
      e45m[i] = f4 - f5;
    }
    const float4 qj = *reinterpret_cast<const float4*>(Cf + PQ + 4 * j);
    const float cj = act ? qj.x : 0.f, dj = act ? qj.y : 0.f;
    const float l2j = Cf[PL2 + j], sj = d0 + l2j;
    const float al = Cf[PA + j], bl = Cf[PB + j], l1l = Cf[PL1 + j];
    float ey[4], ex[4];   // Ey[sa][sc][j] (slot 4 + sa + 2 sc), Ex[sb][sc][j] (slot sb + 2 sc)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ey[q] = W[S::EX + (4 + q) * RS + j];
      ex[q] = W[S::EX + q * RS + j];
    }
    float fc[6], cO[6];   // [4], [5] (z-faces) are read after the walk
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      cO[q] = Cf[PS + q];
      fc[q] = Cf[PS + 6 + q];
    }
    float ze[RS], zo[RS];   // z-contraction over even and over odd k
#pragma unroll
    for (int i = 0; i < RS; ++i) ze[i] = zo[i] = 0.f;
    // line sums along k for the edges, over even and over odd k:
    // sx[2 sa + sc] = sum_k (e|g)_k F_sa[k][j], sy[2 sb + sc] = sum_k (e|g)_k F_{2+sb}[k][i = jl]
    float le[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};   // e_k times A, B, Cl, Dl
    const int ox0 = H[0], ox1 = H[1], oy0 = H[2], oy1 = H[3];

    // ---- walk the y-plane j in k: expansion, D^-1, contractions; x- and
    //      y-face outputs at k
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const float4 qk = *reinterpret_cast<const float4*>(Cf + PQ + 4 * k);
      const float ek = qk.z, gk = qk.w, l3k = Cf[PL3 + k];
      const float4 ezk = *reinterpret_cast<const float4*>(W + S::EZ + 4 * k);   // Ez[sa + 2 sb][k]
      const float A = Fp[k * RS + j], B = Fp[FS + k * RS + j];
      const float Cl = Fp[2 * FS + k * RS + j], Dl = Fp[3 * FS + k * RS + j];
      float Cr[RS], Dr[RS];
      load_row<RS>(Fp + 2 * FS + k * RS, Cr);
      load_row<RS>(Fp + 3 * FS + k * RS, Dr);
      const float sjk = sj + l3k;
      const float ABp = A + B, ABm = A - B;   // a_i A + b_i B = a_i (A +- B)
      float Xe = 0.f, Xo = 0.f;
      float Pr[G];   // c_j D^-1 x along the row
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float x = a[i] * ((i & 1) ? ABm : ABp);
        x = fmaf(cj, Cr[i], x);
        x = fmaf(dj, Dr[i], x);
        x = fmaf(ek, (k & 1) ? e45m[i] : e45p[i], x);   // e_k F4 + g_k F5
        const float w = x * rcp_approx(sjk + l1[i]);   // D^-1 x (the sign is applied at the outputs)
        if (i & 1) Xo = fmaf(a[i], w, Xo);
        else Xe = fmaf(a[i], w, Xe);
        if (k & 1) zo[i] = fmaf(ek, w, zo[i]);
        else ze[i] = fmaf(ek, w, ze[i]);
        Pr[i] = cj * w;
      }
#pragma unroll
      for (int i = N; i < G; ++i) Pr[i] = 0.f;
      const float X0 = Xe + Xo, X1 = Xe - Xo;
      float Y0, Y1;
      reduce_scatter_parity<G>(Pr, jl, &Y0, &Y1);
      if (k & 1) {
        lo[0] = fmaf(ek, A, lo[0]);
        lo[1] = fmaf(ek, B, lo[1]);
        lo[2] = fmaf(ek, Cl, lo[2]);
        lo[3] = fmaf(ek, Dl, lo[3]);
      } else {
        le[0] = fmaf(ek, A, le[0]);
        le[1] = fmaf(ek, B, le[1]);
        le[2] = fmaf(ek, Cl, le[2]);
        le[3] = fmaf(ek, Dl, le[3]);
      }
      if (act) {
        const int kj = k * N + j;
        // x-faces at (k, j): diagonal, opposite face, the four edge lines, -condensed
        const float bx = w0 * (l2j + l3k);
        float o = (fc[0] + bx) * A;
        o = fmaf(cO[0], B, o);
        o = fmaf(w0, fmaf(cj, ezk.x, fmaf(dj, ezk.z, fmaf(ek, ey[0], gk * ey[2]))), o);
        o -= X0;
        if (ox0 >= 0) {
          atomicAdd(v + ox0 + kj, o);
          dot = fmaf(A, o, dot);
        }
        o = (fc[1] + bx) * B;
        o = fmaf(cO[1], A, o);
        o = fmaf(w0, fmaf(cj, ezk.y, fmaf(dj, ezk.w, fmaf(ek, ey[1], gk * ey[3]))), o);
        o -= X1;
        if (ox1 >= 0) {
          atomicAdd(v + ox1 + kj, o);
          dot = fmaf(B, o, dot);
        }
        // y-faces at (k, i = jl)
        const float by = w0 * (l1l + l3k);
        o = (fc[2] + by) * Cl;
        o = fmaf(cO[2], Dl, o);
        o = fmaf(w0, fmaf(al, ezk.x, fmaf(bl, ezk.y, fmaf(ek, ex[0], gk * ex[2]))), o);
        o -= Y0;
        if (oy0 >= 0) {
          atomicAdd(v + oy0 + kj, o);
          dot = fmaf(Cl, o, dot);
        }
        o = (fc[3] + by) * Dl;
        o = fmaf(cO[3], Cl, o);
        o = fmaf(w0, fmaf(al, ezk.z, fmaf(bl, ezk.w, fmaf(ek, ex[1], gk * ex[3]))), o);
        o -= Y1;
        if (oy1 >= 0) {
          atomicAdd(v + oy1 + kj, o);
          dot = fmaf(Dl, o, dot);
        }
      }
    }

    // z-face rows j again, and the even/odd sums combined
    float b[RS], e4[RS], e5[RS];
    cO[4] = Cf[PS + 4];
    cO[5] = Cf[PS + 5];
    fc[4] = Cf[PS + 10];
    fc[5] = Cf[PS + 11];
    load_row<RS>(Cf + PB, b);
    load_row<RS>(Fp + 4 * FS + j * RS, e4);
    load_row<RS>(Fp + 5 * FS + j * RS, e5);
    float (&z4)[RS] = ze;   // in place: z4 = ze + zo, z5 = ze - zo
    float (&z5)[RS] = zo;
#pragma unroll
    for (int i = 0; i < RS; ++i) {
      const float t = ze[i];
      z4[i] = t + zo[i];
      z5[i] = t - z5[i];
    }
    const float sx[4] = {le[0] + lo[0], le[0] - lo[0], le[1] + lo[1], le[1] - lo[1]};
    const float sy[4] = {le[2] + lo[2], le[2] - lo[2], le[3] + lo[3], le[3] - lo[3]};

    // ---- z-faces at (j, i).  The outputs of row j are formed in lane j and
    //      staged in the (no longer needed) z-face rows of shared memory, then
    //      scattered one row per instruction so each atomic row is contiguous.
    float szc[4] = {0.f, 0.f, 0.f, 0.f};   // z-face column l: szc[2 sc + sb] = sum_m (c|d)_m F_{4+sc}[m][l]
    if (act) {
#pragma unroll
      for (int m = 0; m < N; ++m) {
        const float2 cd = *reinterpret_cast<const float2*>(Cf + PQ + 4 * m);
        const float f0 = Fp[4 * FS + m * RS + j], f1 = Fp[5 * FS + m * RS + j];
        szc[0] = fmaf(cd.x, f0, szc[0]);
        szc[1] = fmaf(cd.y, f0, szc[1]);
        szc[2] = fmaf(cd.x, f1, szc[2]);
        szc[3] = fmaf(cd.y, f1, szc[3]);
      }
    }
    __syncwarp();
    const int oz0 = H[4], oz1 = H[5];
    if (act) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        float xa[RS], xb[RS];     // Ex[0][s][.], Ex[1][s][.] (slots 2 s, 2 s + 1)
        load_row<RS>(W + S::EX + (2 * s) * RS, xa);
        load_row<RS>(W + S::EX + (2 * s + 1) * RS, xb);
        const float ya = ey[2 * s], yb = ey[2 * s + 1];   // Ey[0][s][j], Ey[1][s][j]
        float orow[RS];
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const float own = s ? e5[i] : e4[i], opp = s ? e4[i] : e5[i];
          float o = (fc[4 + s] + w0 * (l1[i] + l2j)) * own;
          o = fmaf(cO[4 + s], opp, o);
          o = fmaf(w0, fmaf(a[i], ya, fmaf(b[i], yb, fmaf(cj, xa[i], dj * xb[i]))), o);
          o -= s ? z5[i] : z4[i];
          orow[i] = o;
          dot = fmaf(own, o, dot);   // a Dirichlet face was gathered as zeros: adds 0
        }
#pragma unroll
        for (int i = N; i < RS; ++i) orow[i] = 0.f;
        float* dst = W + S::F + (4 + s) * FS + j * RS;   // row j, 16-byte stores
#pragma unroll
        for (int t = 0; t < RS; t += 4)
          *reinterpret_cast<float4*>(dst + t) = make_float4(orow[t], orow[t + 1], orow[t + 2], orow[t + 3]);
      }
    }
    __syncwarp();
    if (jl < N) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int oz = s ? oz1 : oz0;
        if (oz >= 0) {
#pragma unroll
          for (int t = 0; t < N; ++t) atomicAdd(v + oz + t * N + jl, W[S::F + (4 + s) * FS + t * RS + jl]);
        }
      }
    }
    if (act) {
      // ---- edges at position l = jl
      float szr[4] = {0.f, 0.f, 0.f, 0.f};   // z-face row j: szr[2 sc + sa] = sum_m (a|b)_m F_{4+sc}[j][m]
#pragma unroll
      for (int m = 0; m < N; ++m) {
        szr[0] = fmaf(a[m], e4[m], szr[0]);
        szr[1] = fmaf(b[m], e4[m], szr[1]);
        szr[2] = fmaf(a[m], e5[m], szr[2]);
        szr[3] = fmaf(b[m], e5[m], szr[3]);
      }
      float syr[4] = {0.f, 0.f, 0.f, 0.f};   // y-face row l: syr[2 sb + sa] = sum_m (a|b)_m F_{2+sb}[l][m]
      float sxr[4] = {0.f, 0.f, 0.f, 0.f};   // x-face row l: sxr[2 sa + sb] = sum_m (c|d)_m F_sa[l][m]
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        float yr[RS], xr[RS];
        load_row<RS>(Fp + (2 + f) * FS + j * RS, yr);
        load_row<RS>(Fp + f * FS + j * RS, xr);
#pragma unroll
        for (int m = 0; m < N; ++m) {
          syr[2 * f] = fmaf(a[m], yr[m], syr[2 * f]);
          syr[2 * f + 1] = fmaf(b[m], yr[m], syr[2 * f + 1]);
          const float2 cd = *reinterpret_cast<const float2*>(Cf + PQ + 4 * m);
          sxr[2 * f] = fmaf(cd.x, xr[m], sxr[2 * f]);
          sxr[2 * f + 1] = fmaf(cd.y, xr[m], sxr[2 * f + 1]);
        }
      }
      float Vt[8];
      {
        const float4 v0 = *reinterpret_cast<const float4*>(W + S::VT);
        const float4 v1 = *reinterpret_cast<const float4*>(W + S::VT + 4);
        Vt[0] = v0.x; Vt[1] = v0.y; Vt[2] = v0.z; Vt[3] = v0.w;
        Vt[4] = v1.x; Vt[5] = v1.y; Vt[6] = v1.z; Vt[7] = v1.w;
      }
      const float4 ezl = *reinterpret_cast<const float4*>(W + S::EZ + 4 * j);
      const float ez[4] = {ezl.x, ezl.y, ezl.z, ezl.w};
      const float el = qj.z, gl = qj.w, l3l = Cf[PL3 + j];
      // x-edges Ex[sb][sc] at i = l
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int sb = q & 1, sc = q >> 1;
        float o = (w02 * (d0 + l1l) + Cf[PS + 12 + q]) * ex[q];
        o = fmaf(w02, fmaf(al, Vt[2 * sb + 4 * sc], bl * Vt[1 + 2 * sb + 4 * sc]), o);
        o = fmaf(w0, szc[2 * sc + sb] + sy[2 * sb + sc], o);
        o = fmaf(w0 * cO[2 + sb], ex[(1 - sb) + 2 * sc], o);
        o = fmaf(w0 * cO[4 + sc], ex[sb + 2 * (1 - sc)], o);
        const int off = H[6 + q];
        if (off >= 0) {
          atomicAdd(v + off + j, o);
          dot = fmaf(ex[q], o, dot);
        }
      }
      // y-edges Ey[sa][sc] at j = l
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int sa = q & 1, sc = q >> 1;
        float o = (w02 * (d0 + l2j) + Cf[PS + 16 + q]) * ey[q];
        o = fmaf(w02, fmaf(cj, Vt[sa + 4 * sc], dj * Vt[sa + 2 + 4 * sc]), o);
        o = fmaf(w0, szr[2 * sc + sa] + sx[2 * sa + sc], o);
        o = fmaf(w0 * cO[sa], ey[(1 - sa) + 2 * sc], o);
        o = fmaf(w0 * cO[4 + sc], ey[sa + 2 * (1 - sc)], o);
        const int off = H[10 + q];
        if (off >= 0) {
          atomicAdd(v + off + j, o);
          dot = fmaf(ey[q], o, dot);
        }
      }
      // z-edges Ez[sa][sb] at k = l
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int sa = q & 1, sb = q >> 1;
        float o = (w02 * (d0 + l3l) + Cf[PS + 20 + q]) * ez[q];
        o = fmaf(w02, fmaf(el, Vt[sa + 2 * sb], gl * Vt[sa + 2 * sb + 4]), o);
        o = fmaf(w0, syr[2 * sb + sa] + sxr[2 * sa + sb], o);
        o = fmaf(w0 * cO[sa], ez[(1 - sa) + 2 * sb], o);
        o = fmaf(w0 * cO[2 + sb], ez[sa + 2 * (1 - sb)], o);
        const int off = H[14 + q];
        if (off >= 0) {
          atomicAdd(v + off + j, o);
          dot = fmaf(ez[q], o, dot);
        }
      }
    }
    // ---- vertices (lanes 0..7 of the group, two per lane when G = 4)
    for (int r = jl; r < 8; r += G) {
      const int sa = r & 1, sb = (r >> 1) & 1, sc = r >> 2;
      const float* exr = W + S::EX + (sb + 2 * sc) * RS;
      const float* eyr = W + S::EX + (4 + sa + 2 * sc) * RS;
      float sv = 0.f;
#pragma unroll
      for (int m = 0; m < N; ++m) {
        sv = fmaf(sa ? b[m] : a[m], exr[m], sv);
        sv = fmaf(Cf[PQ + 4 * m + sb], eyr[m], sv);
        sv = fmaf(Cf[PQ + 4 * m + 2 + sc], W[S::EZ + 4 * m + sa + 2 * sb], sv);
      }
      const float vr = W[S::VT + r];
      float o = Cf[PS + 24 + r] * vr;
      o = fmaf(w02, sv, o);
      o = fmaf(w02 * Cf[PS + sa], W[S::VT + (r ^ 1)], o);       // cO from shared memory: the
      o = fmaf(w02 * Cf[PS + 2 + sb], W[S::VT + (r ^ 2)], o);   // index depends on the lane
      o = fmaf(w02 * Cf[PS + 4 + sc], W[S::VT + (r ^ 4)], o);
      const int off = H[18 + r];
      if (off >= 0) {
        atomicAdd(v + off, o);
        dot = fmaf(vr, o, dot);
      }
    }
}

// Per warp, element group after element group ("quads" of EPW elements):
// form the entity offsets, gather by cp.async, compute.  One buffer per
// group slot: a second buffer with the next group's gather in flight
// (a two-stage pipeline) was measured slower (p = 8: 58.7 against 53.6 us
// per application; p = 4: 125 against 120 us): it doubles the CTA's shared
// memory, which the L1 cache gives up, and the other resident warps already
// cover one warp's gather.  v += Hhat~ u over this warp's range of element
// groups; returns the thread's share of u^T v.
template <int N>
__device__ __forceinline__ float plane_apply_all(const SemGeom& g, const SemClassTables<float>& tab,
                                                 const EntityAffine* ent, const float* __restrict__ u,
                                                 float* __restrict__ v, unsigned char* smem_raw) {
  using S = PlaneSm<N>;
  constexpr int G = S::G, EPW = S::EPW;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int grp = lane / G, jl = lane - grp * G;
  const int slot_id = wib * EPW + grp, nslots = wpb * EPW;
  int* H = reinterpret_cast<int*>(smem_raw) + slot_id * kHdr;
  float* W = reinterpret_cast<float*>(smem_raw + (size_t)nslots * kHdr * sizeof(int)) + (size_t)slot_id * S::size;
  // element groups of EPW consecutive elements, split into equal contiguous
  // ranges over all warps of the grid
  const long long nq_all = (g.nelem + EPW - 1) / EPW, nw = (long long)gridDim.x * wpb;
  const long long w = (long long)blockIdx.x * wpb + wib;
  const long long q_begin = nq_all * w / nw;
  const int nq = (int)(nq_all * (w + 1) / nw - q_begin);
  int held = -1;   // class whose coefficient block the slot holds (equal over the group)
  float dot = 0.f;
  for (int qi = 0; qi < nq; ++qi) {
    const long long e = (q_begin + qi) * EPW + grp;
    plane_header<G>(g, tab, ent, (int)e, e < g.nelem, held >= 0 ? held : 0, jl, H);
    __syncwarp();
    const int cls = H[26];
    plane_gather<N>(u, tab.plane + (long long)cls * tab.plane_stride, cls != held, H, W, jl);
    cp_async_commit();
    held = cls;
    cp_async_wait<0>();
    __syncwarp();
    plane_element<N>(W, H, v, jl, dot);
    __syncwarp();
  }
  return dot;
}

template <int N>
__global__ void __launch_bounds__(kPlaneThreads, 4)
k_tpt_apply_plane(SemGeom g, SemClassTables<float> tab, const float* __restrict__ u, float* __restrict__ v,
                  double* __restrict__ partials, PcgState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ EntityAffine ent[26];
  if (st != nullptr && st->done) return;
  if (threadIdx.x < 26) entity_affine(g, threadIdx.x, &ent[threadIdx.x]);
  __syncthreads();
  const float dot = plane_apply_all<N>(g, tab, ent, u, v, smem_raw);
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

// ---------------------------------------------------------------------------
// Two-chunk variant for 9 <= n <= 15: one element per warp, lane (c, j) owns
// the half-row i in [8c, 8c + 8) of y-plane j (16 lanes per half).  The
// x-contraction adds the two halves (one shuffle); the y-contraction is a
// reduce-scatter over the 16 planes of a half (halving on lane bits 2, 1, 0,
// then the pair differing in bit 3), which leaves the sums for position
// l = 8c + (j & 7) on lanes j = 0..7 of half c: those lanes own everything
// indexed by a position (y-face outputs, edges, the line sums along k).
// Face rows are padded to 16 floats and the padding is zero-filled by the
// gather, so the lanes of the short second half compute exact zeros there.
// ---------------------------------------------------------------------------
template <int N>
struct Plane2Sm {
  static constexpr int RS = 16;
  static constexpr int FS = N * RS;
  static constexpr int F = 0;
  static constexpr int EX = 6 * FS;            // x-edges [4][RS], y-edges [4][RS]
  static constexpr int EZ = EX + 8 * RS;       // z-edges [N][4]
  static constexpr int VT = EZ + 4 * N;        // vertices [8]
  static constexpr int C = VT + 8;             // class coefficient block (plane_layout, rs = 16)
  static constexpr int PCS = 5 * RS + 4 * N + 36;
  static constexpr int size = (C + PCS + 3) & ~3;
  static_assert(EZ % 4 == 0 && VT % 4 == 0 && C % 4 == 0, "16-byte alignment");
};

template <int N>
__device__ __forceinline__ void plane2_gather(const float* __restrict__ u, const float* cls_src, bool load_cls,
                                              const int* H, float* W, int lane) {
  using S = Plane2Sm<N>;
  const int half = lane >> 4, col = lane & 15;
#pragma unroll
  for (int slot = 0; slot < 6; ++slot) {
    const int off = H[slot];
#pragma unroll
    for (int rp = 0; rp < N; rp += 2) {
      const int row = rp + half;
      if (row < N) {
        const bool ok = off >= 0 && col < N;
        cp_async4(W + S::F + slot * S::FS + row * S::RS + col, ok ? u + off + row * N + col : u, ok);
      }
    }
  }
#pragma unroll
  for (int sp = 0; sp < 12; sp += 2) {
    const int slot = sp + half, off = H[6 + slot];
    const bool ok = off >= 0 && col < N;
    if (slot < 8) cp_async4(W + S::EX + slot * S::RS + col, ok ? u + off + col : u, ok);
    else if (col < N) cp_async4(W + S::EZ + 4 * col + (slot - 8), ok ? u + off + col : u, ok);
  }
  if (lane < 8) {
    const int off = H[18 + lane];
    cp_async4(W + S::VT + lane, off >= 0 ? u + off : u, off >= 0);
  }
  if (load_cls)
    for (int r = 4 * lane; r < S::PCS; r += 4 * 32) cp_async16(W + S::C + r, cls_src + r);
}

template <int N>
__device__ __forceinline__ void plane2_element(float* W, const int* H, float* __restrict__ v, int lane,
                                               float& dot) {
  using S = Plane2Sm<N>;
  constexpr int RS = S::RS, FS = S::FS;
  constexpr int PA = 0, PB = RS, PL1 = 2 * RS, PL2 = 3 * RS, PL3 = 4 * RS, PQ = 5 * RS, PS = 5 * RS + 4 * N;
  const float* Fp = W + S::F;
  const float* Cf = W + S::C;
  const int c = lane >> 4, jj = lane & 15, i0 = 8 * c;
  const bool actj = jj < N;                   // planes past n mirror plane n-1 and contribute zeros
  const int j = actj ? jj : N - 1;
  const int l = i0 + (jj & 7);                // position owned for y-faces and edges
  const bool actl = jj < 8 && l < N;
  const int lc = l < N ? l : N - 1;           // (lanes jj and jj ^ 8 share the position)

  const float w0 = Cf[PS + 32], w02 = Cf[PS + 33], d0 = Cf[PS + 34];
  float a[8], b[8], l1[8], e4[8], e5[8];
  load_row<8>(Cf + PA + i0, a);
  load_row<8>(Cf + PB + i0, b);
  load_row<8>(Cf + PL1 + i0, l1);
  load_row<8>(Fp + 4 * FS + j * RS + i0, e4);   // z-face rows j, this half
  load_row<8>(Fp + 5 * FS + j * RS + i0, e5);
  const float4 qj = *reinterpret_cast<const float4*>(Cf + PQ + 4 * j);
  const float cj = actj ? qj.x : 0.f, dj = actj ? qj.y : 0.f;
  const float l2j = Cf[PL2 + j], sj = d0 + l2j;
  const float al = Cf[PA + lc], bl = Cf[PB + lc], l1l = Cf[PL1 + lc];
  float ey[4], ex[4];   // Ey[sa][sc][j] (x-faces of plane j), Ex[sb][sc][l] (y-faces, x-edges at l)
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    ey[q] = W[S::EX + (4 + q) * RS + j];
    ex[q] = W[S::EX + q * RS + lc];
  }
  float fc[6], cO[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    cO[q] = Cf[PS + q];
    fc[q] = Cf[PS + 6 + q];
  }
  // the walk's face outputs: lane (c, jj) forms the x-face c output at
  // (k, j) and the y-face jj >> 3 output at (k, l), so every lane forms one
  // output of each kind
  const int fy = jj >> 3;
  const bool actly = l < N;
  const int ox = H[c], oy = H[2 + fy];
  const float fcx = c ? fc[1] : fc[0], cOx = c ? cO[1] : cO[0];   // selects keep the arrays in registers
  const float eyx0 = c ? ey[1] : ey[0], eyx1 = c ? ey[3] : ey[2];
  const float fcy = fy ? fc[3] : fc[2], cOy = fy ? cO[3] : cO[2];
  const float exy0 = fy ? ex[1] : ex[0], exy1 = fy ? ex[3] : ex[2];
  float z4[8], z5[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) z4[t] = z5[t] = 0.f;
  // line sums along k for the edges at l: sx[2 sa + sc] = sum_k (e|g)_k F_sa[k][l],
  // sy[2 sb + sc] = sum_k (e|g)_k F_{2+sb}[k][l]
  float sx[4] = {0.f, 0.f, 0.f, 0.f}, sy[4] = {0.f, 0.f, 0.f, 0.f};

#pragma unroll 1
  for (int k = 0; k < N; ++k) {
    const float4 qk = *reinterpret_cast<const float4*>(Cf + PQ + 4 * k);
    const float ek = qk.z, gk = qk.w, l3k = Cf[PL3 + k];
    const float4 ezk = *reinterpret_cast<const float4*>(W + S::EZ + 4 * k);
    const float A = Fp[k * RS + j], B = Fp[FS + k * RS + j];
    const float Al = Fp[k * RS + lc], Bl = Fp[FS + k * RS + lc];
    const float Cl = Fp[2 * FS + k * RS + lc], Dl = Fp[3 * FS + k * RS + lc];
    float Cr[8], Dr[8];
    load_row<8>(Fp + 2 * FS + k * RS + i0, Cr);
    load_row<8>(Fp + 3 * FS + k * RS + i0, Dr);
    const float sjk = sj + l3k;
    float X0 = 0.f, X1 = 0.f;
    float Wr[8], P0[8], P1[8];   // D^-1 x along the half-row; the partial sums of its y-contraction
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      float x = a[t] * A;
      x = fmaf(b[t], B, x);
      x = fmaf(cj, Cr[t], x);
      x = fmaf(dj, Dr[t], x);
      x = fmaf(ek, e4[t], x);
      x = fmaf(gk, e5[t], x);
      const float w = x * rcp_approx(sjk + l1[t]);
      X0 = fmaf(a[t], w, X0);
      X1 = fmaf(b[t], w, X1);
      z4[t] = fmaf(ek, w, z4[t]);
      z5[t] = fmaf(gk, w, z5[t]);
      Wr[t] = w;
    }
    X0 += __shfl_xor_sync(0xffffffffu, X0, 16);   // both halves of the row
    X1 += __shfl_xor_sync(0xffffffffu, X1, 16);
    halve_w<4, 8>(Wr, cj, dj, P0, P1, jj);
    halve<2, 8>(P0, P1, jj);
    halve<1, 8>(P0, P1, jj);
    const float Y0 = P0[0] + __shfl_xor_sync(0xffffffffu, P0[0], 8);
    const float Y1 = P1[0] + __shfl_xor_sync(0xffffffffu, P1[0], 8);
    sx[0] = fmaf(ek, Al, sx[0]);
    sx[1] = fmaf(gk, Al, sx[1]);
    sx[2] = fmaf(ek, Bl, sx[2]);
    sx[3] = fmaf(gk, Bl, sx[3]);
    sy[0] = fmaf(ek, Cl, sy[0]);
    sy[1] = fmaf(gk, Cl, sy[1]);
    sy[2] = fmaf(ek, Dl, sy[2]);
    sy[3] = fmaf(gk, Dl, sy[3]);
    if (actj) {      // x-face c at (k, j): diagonal, opposite face, the four edge lines, -condensed
      const float own = c ? B : A, opp = c ? A : B;
      float o = (fcx + w0 * (l2j + l3k)) * own;
      o = fmaf(cOx, opp, o);
      o = fmaf(w0, fmaf(cj, c ? ezk.y : ezk.x, fmaf(dj, c ? ezk.w : ezk.z, fmaf(ek, eyx0, gk * eyx1))), o);
      o -= c ? X1 : X0;
      if (ox >= 0) {
        atomicAdd(v + ox + k * N + j, o);
        dot = fmaf(own, o, dot);
      }
    }
    if (actly) {     // y-face jj >> 3 at (k, l)
      const float own = fy ? Dl : Cl, opp = fy ? Cl : Dl;
      float o = (fcy + w0 * (l1l + l3k)) * own;
      o = fmaf(cOy, opp, o);
      o = fmaf(w0, fmaf(al, fy ? ezk.z : ezk.x, fmaf(bl, fy ? ezk.w : ezk.y, fmaf(ek, exy0, gk * exy1))), o);
      o -= fy ? Y1 : Y0;
      if (oy >= 0) {
        atomicAdd(v + oy + k * N + l, o);
        dot = fmaf(own, o, dot);
      }
    }
  }

  // ---- the z-face line sums at l (rows and columns of the z-faces), before
  //      the z-face rows are reused for staging the outputs
  float szr[4] = {0.f, 0.f, 0.f, 0.f};   // z-face row l: szr[2 sc + sa] = sum_m (a|b)_m F_{4+sc}[l][m]
  float szc[4] = {0.f, 0.f, 0.f, 0.f};   // z-face column l: szc[2 sc + sb] = sum_m (c|d)_m F_{4+sc}[m][l]
  if (actl) {
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const float am = Cf[PA + m], bm = Cf[PB + m];
      const float2 cd = *reinterpret_cast<const float2*>(Cf + PQ + 4 * m);
      const float r4 = Fp[4 * FS + l * RS + m], r5 = Fp[5 * FS + l * RS + m];
      const float c4 = Fp[4 * FS + m * RS + l], c5 = Fp[5 * FS + m * RS + l];
      szr[0] = fmaf(am, r4, szr[0]);
      szr[1] = fmaf(bm, r4, szr[1]);
      szr[2] = fmaf(am, r5, szr[2]);
      szr[3] = fmaf(bm, r5, szr[3]);
      szc[0] = fmaf(cd.x, c4, szc[0]);
      szc[1] = fmaf(cd.y, c4, szc[1]);
      szc[2] = fmaf(cd.x, c5, szc[2]);
      szc[3] = fmaf(cd.y, c5, szc[3]);
    }
  }
  __syncwarp();
  // ---- z-faces at (j, i), this half: staged in the z-face rows, then
  //      scattered two rows per instruction
  const int oz0 = H[4], oz1 = H[5];
  if (actj) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      float xa[8], xb[8];     // Ex[0][s][.], Ex[1][s][.] (slots 2 s, 2 s + 1), this half
      load_row<8>(W + S::EX + (2 * s) * RS + i0, xa);
      load_row<8>(W + S::EX + (2 * s + 1) * RS + i0, xb);
      const float ya = ey[2 * s], yb = ey[2 * s + 1];   // Ey[0][s][j], Ey[1][s][j]
      float orow[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const float own = s ? e5[t] : e4[t], opp = s ? e4[t] : e5[t];
        float o = (fc[4 + s] + w0 * (l1[t] + l2j)) * own;
        o = fmaf(cO[4 + s], opp, o);
        o = fmaf(w0, fmaf(a[t], ya, fmaf(b[t], yb, fmaf(cj, xa[t], dj * xb[t]))), o);
        o -= s ? z5[t] : z4[t];
        orow[t] = o;
        dot = fmaf(own, o, dot);   // padding and Dirichlet faces were gathered as zeros: add 0
      }
      float* dst = W + S::F + (4 + s) * FS + j * RS + i0;
      *reinterpret_cast<float4*>(dst) = make_float4(orow[0], orow[1], orow[2], orow[3]);
      *reinterpret_cast<float4*>(dst + 4) = make_float4(orow[4], orow[5], orow[6], orow[7]);
    }
  }
  __syncwarp();
  {
    const int half = lane >> 4, col = lane & 15;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int oz = s ? oz1 : oz0;
      if (oz >= 0 && col < N) {
#pragma unroll
        for (int rp = 0; rp < N; rp += 2) {
          const int row = rp + half;
          if (row < N) atomicAdd(v + oz + row * N + col, W[S::F + (4 + s) * FS + row * RS + col]);
        }
      }
    }
  }
  // ---- edges at position l
  if (actl) {
    float syr[4] = {0.f, 0.f, 0.f, 0.f};   // y-face row l: syr[2 sb + sa] = sum_m (a|b)_m F_{2+sb}[l][m]
    float sxr[4] = {0.f, 0.f, 0.f, 0.f};   // x-face row l: sxr[2 sa + sb] = sum_m (c|d)_m F_sa[l][m]
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const float am = Cf[PA + m], bm = Cf[PB + m];
      const float2 cd = *reinterpret_cast<const float2*>(Cf + PQ + 4 * m);
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        const float yr = Fp[(2 + f) * FS + l * RS + m], xr = Fp[f * FS + l * RS + m];
        syr[2 * f] = fmaf(am, yr, syr[2 * f]);
        syr[2 * f + 1] = fmaf(bm, yr, syr[2 * f + 1]);
        sxr[2 * f] = fmaf(cd.x, xr, sxr[2 * f]);
        sxr[2 * f + 1] = fmaf(cd.y, xr, sxr[2 * f + 1]);
      }
    }
    float Vt[8];
    {
      const float4 v0 = *reinterpret_cast<const float4*>(W + S::VT);
      const float4 v1 = *reinterpret_cast<const float4*>(W + S::VT + 4);
      Vt[0] = v0.x; Vt[1] = v0.y; Vt[2] = v0.z; Vt[3] = v0.w;
      Vt[4] = v1.x; Vt[5] = v1.y; Vt[6] = v1.z; Vt[7] = v1.w;
    }
    const float4 ezl = *reinterpret_cast<const float4*>(W + S::EZ + 4 * l);
    const float ez[4] = {ezl.x, ezl.y, ezl.z, ezl.w};
    const float4 ql = *reinterpret_cast<const float4*>(Cf + PQ + 4 * l);
    const float l2l = Cf[PL2 + l], l3l = Cf[PL3 + l];
    float eyl[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) eyl[q] = W[S::EX + (4 + q) * RS + l];
    // x-edges Ex[sb][sc] at i = l
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int sb = q & 1, sc = q >> 1;
      float o = (w02 * (d0 + l1l) + Cf[PS + 12 + q]) * ex[q];
      o = fmaf(w02, fmaf(al, Vt[2 * sb + 4 * sc], bl * Vt[1 + 2 * sb + 4 * sc]), o);
      o = fmaf(w0, szc[2 * sc + sb] + sy[2 * sb + sc], o);
      o = fmaf(w0 * cO[2 + sb], ex[(1 - sb) + 2 * sc], o);
      o = fmaf(w0 * cO[4 + sc], ex[sb + 2 * (1 - sc)], o);
      const int off = H[6 + q];
      if (off >= 0) {
        atomicAdd(v + off + l, o);
        dot = fmaf(ex[q], o, dot);
      }
    }
    // y-edges Ey[sa][sc] at j = l
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int sa = q & 1, sc = q >> 1;
      float o = (w02 * (d0 + l2l) + Cf[PS + 16 + q]) * eyl[q];
      o = fmaf(w02, fmaf(ql.x, Vt[sa + 4 * sc], ql.y * Vt[sa + 2 + 4 * sc]), o);
      o = fmaf(w0, szr[2 * sc + sa] + sx[2 * sa + sc], o);
      o = fmaf(w0 * cO[sa], eyl[(1 - sa) + 2 * sc], o);
      o = fmaf(w0 * cO[4 + sc], eyl[sa + 2 * (1 - sc)], o);
      const int off = H[10 + q];
      if (off >= 0) {
        atomicAdd(v + off + l, o);
        dot = fmaf(eyl[q], o, dot);
      }
    }
    // z-edges Ez[sa][sb] at k = l
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int sa = q & 1, sb = q >> 1;
      float o = (w02 * (d0 + l3l) + Cf[PS + 20 + q]) * ez[q];
      o = fmaf(w02, fmaf(ql.z, Vt[sa + 2 * sb], ql.w * Vt[sa + 2 * sb + 4]), o);
      o = fmaf(w0, syr[2 * sb + sa] + sxr[2 * sa + sb], o);
      o = fmaf(w0 * cO[sa], ez[(1 - sa) + 2 * sb], o);
      o = fmaf(w0 * cO[2 + sb], ez[sa + 2 * (1 - sb)], o);
      const int off = H[14 + q];
      if (off >= 0) {
        atomicAdd(v + off + l, o);
        dot = fmaf(ez[q], o, dot);
      }
    }
  }
  // ---- vertices (lanes 0..7)
  if (lane < 8) {
    const int r = lane, sa = r & 1, sb = (r >> 1) & 1, sc = r >> 2;
    const float* exr = W + S::EX + (sb + 2 * sc) * RS;
    const float* eyr = W + S::EX + (4 + sa + 2 * sc) * RS;
    float sv = 0.f;
#pragma unroll
    for (int m = 0; m < N; ++m) {
      sv = fmaf(Cf[(sa ? PB : PA) + m], exr[m], sv);
      sv = fmaf(Cf[PQ + 4 * m + sb], eyr[m], sv);
      sv = fmaf(Cf[PQ + 4 * m + 2 + sc], W[S::EZ + 4 * m + sa + 2 * sb], sv);
    }
    const float vr = W[S::VT + r];
    float o = Cf[PS + 24 + r] * vr;
    o = fmaf(w02, sv, o);
    o = fmaf(w02 * Cf[PS + sa], W[S::VT + (r ^ 1)], o);
    o = fmaf(w02 * Cf[PS + 2 + sb], W[S::VT + (r ^ 2)], o);
    o = fmaf(w02 * Cf[PS + 4 + sc], W[S::VT + (r ^ 4)], o);
    const int off = H[18 + r];
    if (off >= 0) {
      atomicAdd(v + off, o);
      dot = fmaf(vr, o, dot);
    }
  }
}

// One element per warp; a two-stage gather pipeline: while one element is
// computed, the next element's offsets are formed and its gather is in flight
// into a second buffer (measured faster here than one buffer, unlike the
// one-row kernel above).  v += Hhat~ u; returns the thread's share of u^T v.
template <int N>
__device__ __forceinline__ float plane2_apply_all(const SemGeom& g, const SemClassTables<float>& tab,
                                                  const EntityAffine* ent, const float* __restrict__ u,
                                                  float* __restrict__ v, unsigned char* smem_raw) {
  using S = Plane2Sm<N>;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  int* H0 = reinterpret_cast<int*>(smem_raw) + wib * kHdr;
  float* W0 = reinterpret_cast<float*>(smem_raw + (size_t)2 * wpb * kHdr * sizeof(int)) + (size_t)wib * S::size;
  const int hstep = wpb * kHdr, wstep = wpb * S::size;
  const long long ne = g.nelem, nw = (long long)gridDim.x * wpb;
  const long long w = (long long)blockIdx.x * wpb + wib;
  const long long e_begin = ne * w / nw;
  const int ncount = (int)(ne * (w + 1) / nw - e_begin);
  int held0 = -1, held1 = -1;
  float dot = 0.f;
  auto stage = [&](int qi, int b) {
    int* H = H0 + b * hstep;
    float* W = W0 + b * wstep;
    const int held = b ? held1 : held0;
    const long long e = e_begin + qi;
    plane_header<32>(g, tab, ent, (int)e, e < ne, held >= 0 ? held : 0, lane, H);
    __syncwarp();
    const int cls = H[26];
    plane2_gather<N>(u, tab.plane + (long long)cls * tab.plane_stride, cls != held, H, W, lane);
    cp_async_commit();
    if (b) held1 = cls;
    else held0 = cls;
  };
  if (ncount > 0) stage(0, 0);
  for (int qi = 0; qi < ncount; ++qi) {
    const int b = qi & 1;
    if (qi + 1 < ncount) {
      stage(qi + 1, b ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    plane2_element<N>(W0 + b * wstep, H0 + b * hstep, v, lane, dot);
    __syncwarp();
  }
  return dot;
}

template <int N>
__global__ void __launch_bounds__(kPlaneThreads, 4)
k_tpt_apply_plane2(SemGeom g, SemClassTables<float> tab, const float* __restrict__ u, float* __restrict__ v,
                   double* __restrict__ partials, PcgState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ EntityAffine ent[26];
  if (st != nullptr && st->done) return;
  if (threadIdx.x < 26) entity_affine(g, threadIdx.x, &ent[threadIdx.x]);
  __syncthreads();
  const float dot = plane2_apply_all<N>(g, tab, ent, u, v, smem_raw);
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
void launch_plane2_n(const SemGeom& g, const SemClassTables<float>& t, const float* x, float* y, double* partials,
                     PcgState* st, cudaStream_t s) {
  using S = Plane2Sm<N>;
  const int wpb = kPlaneThreads / 32;
  const size_t smem = (size_t)2 * wpb * kHdr * sizeof(int) + (size_t)2 * wpb * S::size * sizeof(float);
  static bool attr = false;
  if (!attr) {   // once per instantiation; the first launch happens outside any capture
    cudaFuncSetAttribute(k_tpt_apply_plane2<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tpt_apply_plane2<N>, kPlaneThreads, smem);
  if (occ < 1) occ = 1;
  long long grid = (long long)sem_num_sms() * occ;
  const long long need = (g.nelem + wpb - 1) / wpb;
  if (grid > need) grid = need;
  k_tpt_apply_plane2<N><<<(int)grid, kPlaneThreads, smem, s>>>(g, t, x, y, partials, st);
  sem_count_launch();
}

template <int N>
size_t plane_smem() {
  using S = PlaneSm<N>;
  const int wpb = kPlaneThreads / 32;
  return (size_t)wpb * S::EPW * kHdr * sizeof(int) + (size_t)wpb * S::EPW * S::size * sizeof(float);
}

template <int N>
void launch_plane_n(const SemGeom& g, const SemClassTables<float>& t, const float* x, float* y, double* partials,
                    PcgState* st, cudaStream_t s) {
  using S = PlaneSm<N>;
  const int wpb = kPlaneThreads / 32;
  const size_t smem = plane_smem<N>();
  static bool attr = false;
  if (!attr) {   // once per instantiation; the first launch happens outside any capture
    cudaFuncSetAttribute(k_tpt_apply_plane<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tpt_apply_plane<N>, kPlaneThreads, smem);
  if (occ < 1) occ = 1;
  // one full wave of resident blocks (fewer if there are fewer element groups than warps)
  const long long nq = (g.nelem + S::EPW - 1) / S::EPW;
  long long grid = (long long)sem_num_sms() * occ;
  const long long need = (nq + wpb - 1) / wpb;
  if (grid > need) grid = need;
  k_tpt_apply_plane<N><<<(int)grid, kPlaneThreads, smem, s>>>(g, t, x, y, partials, st);
  sem_count_launch();
}

// Class blocks in the layout of plane_layout(n), from the metric
// coefficients d0..d3 of each class and the 1D basis (FP64, stored in FP32).
__global__ void k_plane_coeffs(SemGeom g, SemBasis b, const double* __restrict__ dcoef, float* __restrict__ out) {
  const int n = g.n;
  const PlaneLayout L = plane_layout(n);
  const long long ncls = (long long)g.ux * g.uy * g.uz;
  const double w0 = b.w0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncls * L.stride;
       t += (long long)gridDim.x * blockDim.x) {
    const long long c = t / L.stride;
    const int r = (int)(t - c * L.stride);
    const double* d = dcoef + c * 4;
    double val = 0.0;
    if (r < L.pq) {
      const int row = r / L.rs, i = r - row * L.rs;
      if (i < n) {
        if (row == 0) val = d[1] * b.k[0][i];
        else if (row == 1) val = d[1] * b.k[1][i];
        else val = d[row - 1] * b.lam[i];        // rows 2, 3, 4: d1, d2, d3 times lambda
      }
    } else if (r < L.ps) {
      const int m = (r - L.pq) >> 2, comp = (r - L.pq) & 3;
      val = d[comp < 2 ? 2 : 3] * b.k[comp & 1][m];
    } else {
      const int q = r - L.ps;
      if (q < 6) {                                // cO
        const int dir = q >> 1, s = q & 1;
        val = d[dir + 1] * b.K[s][1 - s];
      } else if (q < 12) {                        // face-diagonal constants
        const int slot = q - 6, dir = slot >> 1, s = slot & 1;
        val = d[0] * w0 + d[dir + 1] * b.K[s][s];
      } else if (q < 24) {                        // edge-diagonal constants
        const int slot = q - 12, grp = slot >> 2, s1 = slot & 1, s2 = (slot >> 1) & 1;
        const int t1 = grp == 0 ? 1 : 0, t2 = grp == 2 ? 1 : 2;
        val = w0 * (d[t1 + 1] * b.K[s1][s1] + d[t2 + 1] * b.K[s2][s2]);
      } else if (q < 32) {                        // vertex diagonals
        const int slot = q - 24, sa = slot & 1, sb = (slot >> 1) & 1, sc = slot >> 2;
        val = d[0] * w0 * w0 * w0 + w0 * w0 * (d[1] * b.K[sa][sa] + d[2] * b.K[sb][sb] + d[3] * b.K[sc][sc]);
      } else if (q == 32) {
        val = w0;
      } else if (q == 33) {
        val = w0 * w0;
      } else if (q == 34) {
        val = d[0];
      }
    }
    out[t] = (float)val;
  }
}

}  // namespace

void launch_plane_coeffs(const SemGeom& g, const SemBasis& b, const double* dcoef, float* plane, cudaStream_t s) {
  const long long work = (long long)g.ux * g.uy * g.uz * plane_layout(g.n).stride;
  long long blocks = (work + 255) / 256;
  if (blocks > (long long)sem_num_sms() * 16) blocks = (long long)sem_num_sms() * 16;
  if (blocks < 1) blocks = 1;
  k_plane_coeffs<<<(int)blocks, 256, 0, s>>>(g, b, dcoef, plane);
  sem_count_launch();
}

void launch_plane_apply(const SemGeom& g, const SemClassTables<float>& t, const float* x, float* y,
                        double* partials, PcgState* st, cudaStream_t s) {
  switch (g.n) {
    case 9: launch_plane2_n<9>(g, t, x, y, partials, st, s); return;
    case 10: launch_plane2_n<10>(g, t, x, y, partials, st, s); return;
    case 11: launch_plane2_n<11>(g, t, x, y, partials, st, s); return;
    case 12: launch_plane2_n<12>(g, t, x, y, partials, st, s); return;
    case 13: launch_plane2_n<13>(g, t, x, y, partials, st, s); return;
    case 14: launch_plane2_n<14>(g, t, x, y, partials, st, s); return;
    case 15: launch_plane2_n<15>(g, t, x, y, partials, st, s); return;
    default: break;
  }
  switch (g.n) {
    case 2: launch_plane_n<2>(g, t, x, y, partials, st, s); break;
    case 3: launch_plane_n<3>(g, t, x, y, partials, st, s); break;
    case 4: launch_plane_n<4>(g, t, x, y, partials, st, s); break;
    case 5: launch_plane_n<5>(g, t, x, y, partials, st, s); break;
    case 6: launch_plane_n<6>(g, t, x, y, partials, st, s); break;
    case 7: launch_plane_n<7>(g, t, x, y, partials, st, s); break;
    default: launch_plane_n<8>(g, t, x, y, partials, st, s); break;
  }
}

SEM_DEBUG_TU(plane)
