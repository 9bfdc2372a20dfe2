// k-slab variant of the transformed condensed operator (Sec. 6 of the paper)
// for FP32 and 16 <= n <= 31: the inner operator of the mixed-precision solve
// at high degree.
//
// The element operator is the one of the other variants (sem_apply.cu,
// sem_apply_plane.cu): the six faces expanded into the interior eigenspace
// (Table 2), D^-1 (Eq. hii_diagonal), the contraction back onto the faces,
// and the primary part H~_BB restricted to the skeleton.  Only the mapping of
// the work onto the GPU differs.
//
// * A work unit is one element and one slab of K = 8 planes k of its n^3
//   eigenspace cube; a CTA of four warps takes one unit (a range of units
//   past 65536 of them).  The
//   expansion and D^-1 are pointwise in k, so a slab's share of the x- and
//   y-face outputs is complete (their rows k in the slab) and its share of
//   the z-face outputs (sums over k) is a partial sum, added by the scatter
//   like the neighbour element's.  At p = 32 an 8^3 mesh gives 2048 units
//   for 152 SMs instead of 512 elements.
// * Thread (j, c) holds the chunk i in [8c, 8c + 8) of row j and walks the
//   slab in k.  The z-contraction (over k) stays in its registers; the
//   x-contraction (over i) is eight register terms and a reduce-scatter over
//   the four chunk lanes; the y-contraction (over j) goes through shared
//   memory: the slab of D^-1 x is stored, then each thread sums one block of
//   (k, 4 i) over half of the j range and the halves are added by a shuffle.
// * D^-1 = 1 / (d0 + d1 lambda_i + d2 lambda_j + d3 lambda_k) is formed per
//   point with one reciprocal (as in the plane kernels), from the class block
//   of plane_layout(n).
// * The primary part of each face output is formed by the thread that holds
//   its operands (the walk thread for the x- and z-faces, the y-contraction
//   thread for the y-faces).  Line sums of the primary part that run along k
//   are split over the slabs in the same way as the condensed sums; the rest
//   of the primary part is done once per element (the z-face rows by a 1 / S
//   share per slab, edges and vertices by slab 0).
// * Outputs are staged in shared memory and scattered one row per warp
//   instruction (contiguous red.global.add).
#include <cuda_runtime.h>

#include "sem_device.cuh"
#include "sem_kernels.cuh"

using namespace semdev;

namespace {

constexpr int kSlabThreads = 128;
constexpr int kK = 8;     // planes k per work unit
constexpr int kR = 32;    // padded row (i or j): n <= 31
constexpr int kZ = kR * kR;

// Shared-memory layout (floats).  Rows of 32; the z-faces and the slab swizzle
// the 16-byte chunks of row j by (j & 7), so that eight rows read or written
// at the same chunk fall into different banks.
struct SlabSm {
  static constexpr int FX = 0;                  // x-faces, rows k of the slab [2][K][32] (kk, j)
  static constexpr int FY = FX + 2 * kK * kR;   // y-faces, rows k of the slab [2][K][32] (kk, i)
  static constexpr int FZ = FY + 2 * kK * kR;   // z-faces [2][32][32] (j, i), swizzled
  static constexpr int EXY = FZ + 2 * kZ;       // x-edges [4][32] (sb + 2 sc), y-edges [4][32] (4 + sa + 2 sc)
  static constexpr int EZ = EXY + 8 * kR;       // z-edges [32][4] (k; component sa + 2 sb)
  static constexpr int VT = EZ + 4 * kR;        // vertices [8]
  static constexpr int CA = VT + 8;             // a_i = d1 k0[i]              [32], 0 past n
  static constexpr int CB = CA + kR;            // b_i = d1 k1[i]              [32], 0 past n
  static constexpr int CL1 = CB + kR;           // d1 lambda_i                 [32], 1 past n
  static constexpr int CL2 = CL1 + kR;          // d2 lambda_j                 [32], 1 past n
  static constexpr int CCD = CL2 + kR;          // (c_j, d_j) = d2 (k0, k1)[j] [32][2], 0 past n
  static constexpr int CEG = CCD + 2 * kR;      // (e_k, g_k, d3 lambda_k, 0)  [32][4], (0, 0, 1, 0) past n
  static constexpr int CPS = CEG + 4 * kR;      // scalars of the class block (plane_layout ps) [36]
  static constexpr int V = CPS + 40;            // slab of D^-1 x [K][32][32] (kk, j, i), swizzled;
                                                // then the z-face sums [2][32][32] (j, i), swizzled
  static constexpr int OX = V + kK * kZ;        // x-face condensed sums [2][K][32] (kk, j)
  static constexpr int OY = OX + 2 * kK * kR;   // y-face condensed sums [2][K][32] (kk, i)
  static constexpr int HDR = OY + 2 * kK * kR;  // ints: 26 entity offsets, class
  static constexpr int size = HDR + 32;
  static_assert(CA % 4 == 0 && CCD % 4 == 0 && CEG % 4 == 0 && V % 4 == 0 && OY % 4 == 0, "16-byte alignment");
};

// Position of (row j, column i) in a swizzled 32 x 32 block.
__device__ __forceinline__ int swz(int j, int i) { return j * kR + ((((i >> 2) ^ (j & 7)) << 2) | (i & 3)); }

// The 8 floats i in [8c, 8c + 8) of row j of a swizzled block.
__device__ __forceinline__ void load_chunk(const float* blk, int j, int c, float (&r)[8]) {
  const float* row = blk + j * kR;
  const float4 v0 = *reinterpret_cast<const float4*>(row + (((2 * c) ^ (j & 7)) << 2));
  const float4 v1 = *reinterpret_cast<const float4*>(row + (((2 * c + 1) ^ (j & 7)) << 2));
  r[0] = v0.x; r[1] = v0.y; r[2] = v0.z; r[3] = v0.w;
  r[4] = v1.x; r[5] = v1.y; r[6] = v1.z; r[7] = v1.w;
}
__device__ __forceinline__ void store_chunk(float* blk, int j, int c, const float (&r)[8]) {
  float* row = blk + j * kR;
  *reinterpret_cast<float4*>(row + (((2 * c) ^ (j & 7)) << 2)) = make_float4(r[0], r[1], r[2], r[3]);
  *reinterpret_cast<float4*>(row + (((2 * c + 1) ^ (j & 7)) << 2)) = make_float4(r[4], r[5], r[6], r[7]);
}
// 8 floats from a 16-byte aligned row.
__device__ __forceinline__ void load8(const float* p, float (&r)[8]) {
  const float4 v0 = *reinterpret_cast<const float4*>(p);
  const float4 v1 = *reinterpret_cast<const float4*>(p + 4);
  r[0] = v0.x; r[1] = v0.y; r[2] = v0.z; r[3] = v0.w;
  r[4] = v1.x; r[5] = v1.y; r[6] = v1.z; r[7] = v1.w;
}

// Entity offsets of element e (-1 on the Dirichlet boundary) and its class.
__device__ __forceinline__ void slab_header(const SemGeom& g, const SemClassTables<float>& tab,
                                            const EntityAffine* ent, int e, int r, int* H) {
  const int mxy = g.mx * g.my, ez = e / mxy, rem = e - ez * mxy, ey = rem / g.mx, ex = rem - ey * g.mx;
  if (r == 26) {
    H[26] = elem_class(g, tab, ex, ey, ez);
  } else {
    const int bits = (ex == 0) | ((ex == g.mx - 1) << 1) | ((ey == 0) << 2) | ((ey == g.my - 1) << 3) |
                     ((ez == 0) << 4) | ((ez == g.mz - 1) << 5);
    const EntityAffine a = ent[r];
    H[r] = entity_offset(a, r, bits, ex, ey, ez, g);
  }
}

// Gather R^T of the unit's data (cp.async, zero-filled past n and on
// Dirichlet entities) and the class coefficients with the padding the walk
// needs.
__device__ __forceinline__ void slab_gather(const SemGeom& g, const SemClassTables<float>& tab,
                                            const float* __restrict__ u, const int* H, int k0, float* sm) {
  using S = SlabSm;
  const int n = g.n, tid = threadIdx.x, x = tid & 31, row = tid >> 5;
  const bool xin = x < n;
  // item t = tid + 128 r of each loop: the lane is the position in the row,
  // the warp and r name the row
#pragma unroll
  for (int r = 0; r < 8; ++r) {   // x- and y-face rows of the slab (slots 0..3): [slot][kk][x]
    const int slot = r >> 1, kk = row + 4 * (r & 1), k = k0 + kk;
    const int off = H[slot];
    const bool ok = off >= 0 && k < n && xin;
    cp_async4(sm + S::FX + tid + 128 * r, ok ? u + off + k * n + x : u, ok);
  }
  const int col0 = (((x >> 2) ^ (row & 7)) << 2) | (x & 3);          // swizzled column, rows j = row + 8 t
  const int col1 = (((x >> 2) ^ ((row + 4) & 7)) << 2) | (x & 3);    // rows j = row + 4 + 8 t
#pragma unroll 2
  for (int r = 0; r < 16; ++r) {  // z-faces (slots 4, 5): [f][j][x], j = row + 4 (r & 7)
    const int f = r >> 3, j = row + 4 * (r & 7);
    const int off = H[4 + f];
    const bool ok = off >= 0 && j < n && xin;
    cp_async4(sm + S::FZ + f * kZ + j * kR + ((r & 1) ? col1 : col0), ok ? u + off + j * n + x : u, ok);
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {   // edges (slots 6..17), slot 6 + q with q = row + 4 r
    const int q = row + 4 * r;
    const int off = H[6 + q];
    const bool ok = off >= 0 && xin;
    float* dst = r < 2 ? sm + S::EXY + q * kR + x : sm + S::EZ + 4 * x + (q - 8);
    cp_async4(dst, ok ? u + off + x : u, ok);
  }
  if (tid < 8) {                                              // vertices (slots 18..25)
    const int off = H[18 + tid];
    cp_async4(sm + S::VT + tid, off >= 0 ? u + off : u, off >= 0);
  }
  cp_async_commit();
  const PlaneLayout L = plane_layout(n);
  const float* cb = tab.plane + (long long)H[26] * tab.plane_stride;
  if (tid < kR) {
    const int m = tid;
    const bool in = m < n;
    sm[S::CA + m] = in ? cb[L.pa + m] : 0.f;
    sm[S::CB + m] = in ? cb[L.pb + m] : 0.f;
    sm[S::CL1 + m] = in ? cb[L.pl1 + m] : 1.f;
    sm[S::CL2 + m] = in ? cb[L.pl2 + m] : 1.f;
    const float4 q = in ? *reinterpret_cast<const float4*>(cb + L.pq + 4 * m) : make_float4(0.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float2*>(sm + S::CCD + 2 * m) = make_float2(q.x, q.y);
    *reinterpret_cast<float4*>(sm + S::CEG + 4 * m) = make_float4(q.z, q.w, in ? cb[L.pl3 + m] : 1.f, 0.f);
  } else if (tid < kR + 36) {
    sm[S::CPS + tid - kR] = cb[L.ps + tid - kR];
  }
}

// The faces of one unit: the walk over the slab (x- and z-contractions,
// D^-1 x stored), the y-contraction from shared memory, and the primary part
// of each face output, formed by the thread that holds its operands (the walk
// thread for the x- and z-faces, the y-contraction thread for the y-faces).
// Leaves the finished outputs (primary minus condensed) in OX / OY and, for
// the z-faces (the slab's partial sums), in the slab area; adds their share
// of x^T (A x) to dot (inputs past n or on Dirichlet faces were gathered as
// zeros, so those terms add 0).
__device__ __forceinline__ void slab_faces(const SemGeom& g, int s, int nslab, int k0, float* sm, float& dot) {
  using S = SlabSm;
  const int n = g.n, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int jl = lane & 7, c = lane >> 3, j = 8 * w + jl, i0 = 8 * c;
  const float w0 = sm[S::CPS + 32], d0 = sm[S::CPS + 34];
  float zb[8], zt[8];
  {
    float a[8], b[8], l1[8], zi0[8], zi1[8];
    load8(sm + S::CA + i0, a);
    load8(sm + S::CB + i0, b);
    load8(sm + S::CL1 + i0, l1);
    load_chunk(sm + S::FZ, j, c, zi0);
    load_chunk(sm + S::FZ + kZ, j, c, zi1);
    const float2 cd = *reinterpret_cast<const float2*>(sm + S::CCD + 2 * j);
    const float cj = cd.x, dj = cd.y, l2j = sm[S::CL2 + j], sj = d0 + l2j;
    float X[2 * kK];
#pragma unroll
    for (int t = 0; t < 8; ++t) zb[t] = zt[t] = 0.f;
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) {
      const float4 eg = *reinterpret_cast<const float4*>(sm + S::CEG + 4 * (k0 + kk));
      const float A = sm[S::FX + kk * kR + j], B = sm[S::FX + (kK + kk) * kR + j];
      float cr[8], dr[8], wr[8];
      load8(sm + S::FY + kk * kR + i0, cr);
      load8(sm + S::FY + (kK + kk) * kR + i0, dr);
      const float sjk = sj + eg.z;
      float x0 = 0.f, x1 = 0.f;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        float x = a[t] * A;
        x = fmaf(b[t], B, x);
        x = fmaf(cj, cr[t], x);
        x = fmaf(dj, dr[t], x);
        x = fmaf(eg.x, zi0[t], x);
        x = fmaf(eg.y, zi1[t], x);
        const float wv = x * rcp_approx(sjk + l1[t]);   // D^-1 x (the sign is applied at the outputs)
        x0 = fmaf(a[t], wv, x0);
        x1 = fmaf(b[t], wv, x1);
        zb[t] = fmaf(eg.x, wv, zb[t]);
        zt[t] = fmaf(eg.y, wv, zt[t]);
        wr[t] = wv;
      }
      X[kk] = x0;
      X[kK + kk] = x1;
      store_chunk(sm + S::V + kk * kZ, j, c, wr);
    }
    // x-contraction over the four chunks of row j (lane bits 4 and 3): a
    // reduce-scatter that leaves face c >> 1, planes 4 (c & 1) .. + 3 on lane c
    {
      const bool up = (lane & 16) != 0;
#pragma unroll
      for (int t = 0; t < kK; ++t) {
        const float snd = up ? X[t] : X[t + kK], kp = up ? X[t + kK] : X[t];
        X[t] = kp + __shfl_xor_sync(0xffffffffu, snd, 16);
      }
    }
    {
      const bool up = (lane & 8) != 0;
#pragma unroll
      for (int t = 0; t < kK / 2; ++t) {
        const float snd = up ? X[t] : X[t + kK / 2], kp = up ? X[t + kK / 2] : X[t];
        X[t] = kp + __shfl_xor_sync(0xffffffffu, snd, 8);
      }
    }
    // x-face outputs at (k, j), face f: diagonal, opposite face, the four edge
    // lines, minus the condensed sum
    {
      const int f = c >> 1, kb = 4 * (c & 1);
      const float ey0 = sm[S::EXY + (4 + f) * kR + j], ey1 = sm[S::EXY + (6 + f) * kR + j];   // Ey[f][0|1] at j
      const float fcx = sm[S::CPS + 6 + f], cOx = sm[S::CPS + f];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int kk = kb + t, k = k0 + kk;
        const float A = sm[S::FX + (f * kK + kk) * kR + j], B = sm[S::FX + ((1 - f) * kK + kk) * kR + j];
        const float4 eg = *reinterpret_cast<const float4*>(sm + S::CEG + 4 * k);
        const float ez0 = sm[S::EZ + 4 * k + f], ez1 = sm[S::EZ + 4 * k + 2 + f];   // Ez[f][0|1] at k
        float o = (fcx + w0 * (l2j + eg.z)) * A;
        o = fmaf(cOx, B, o);
        o = fmaf(w0, fmaf(cj, ez0, fmaf(dj, ez1, fmaf(eg.x, ey0, eg.y * ey1))), o);
        o -= X[t];
        sm[S::OX + (f * kK + kk) * kR + j] = o;
        dot = fmaf(A, o, dot);
      }
    }
    // z-face outputs at (j, i in the chunk): the primary part of rows
    // [jlo, jhi) (a 1 / S share) minus the slab's condensed sums
    const int jrows = (n + nslab - 1) / nslab, jlo = s * jrows;
    if (j >= jlo && j < jlo + jrows) {
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        const float ya = sm[S::EXY + (4 + 2 * f) * kR + j], yb = sm[S::EXY + (5 + 2 * f) * kR + j];   // Ey[0|1][f] at j
        float xa[8], xb[8];                                                                           // Ex[0|1][f] at i
        load8(sm + S::EXY + (2 * f) * kR + i0, xa);
        load8(sm + S::EXY + (1 + 2 * f) * kR + i0, xb);
        const float fcz = sm[S::CPS + 10 + f] + w0 * l2j, cOz = sm[S::CPS + 4 + f];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const float own = f ? zi1[t] : zi0[t], opp = f ? zi0[t] : zi1[t];
          float o = fmaf(w0, l1[t], fcz) * own;
          o = fmaf(cOz, opp, o);
          o = fmaf(w0, fmaf(a[t], ya, fmaf(b[t], yb, fmaf(cj, xa[t], dj * xb[t]))), o);
          if (f) zt[t] = o - zt[t];
          else zb[t] = o - zb[t];
        }
      }
    } else {
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        zb[t] = -zb[t];
        zt[t] = -zt[t];
      }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) dot = fmaf(zi0[t], zb[t], fmaf(zi1[t], zt[t], dot));
  }
  __syncthreads();
  // y-contraction: thread (kk, iq, jh) sums (c_j, d_j) times the slab over
  // j in [16 jh, 16 jh + 16) for i in [4 iq, 4 iq + 4); then the y-face
  // outputs of face jh at (k, i)
  {
    const int iq = lane & 7, jh = (lane >> 3) & 1, kk = (lane >> 4) + 2 * w, k = k0 + kk, i = 4 * iq;
    float s0[4] = {0.f, 0.f, 0.f, 0.f}, s1[4] = {0.f, 0.f, 0.f, 0.f};
    const float* slab = sm + S::V + kk * kZ;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int jj = 16 * jh + t;
      const float4 vv = *reinterpret_cast<const float4*>(slab + jj * kR + ((iq ^ (jj & 7)) << 2));
      const float2 cd = *reinterpret_cast<const float2*>(sm + S::CCD + 2 * jj);
      s0[0] = fmaf(cd.x, vv.x, s0[0]);
      s0[1] = fmaf(cd.x, vv.y, s0[1]);
      s0[2] = fmaf(cd.x, vv.z, s0[2]);
      s0[3] = fmaf(cd.x, vv.w, s0[3]);
      s1[0] = fmaf(cd.y, vv.x, s1[0]);
      s1[1] = fmaf(cd.y, vv.y, s1[1]);
      s1[2] = fmaf(cd.y, vv.z, s1[2]);
      s1[3] = fmaf(cd.y, vv.w, s1[3]);
    }
    float y[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {   // half jh keeps face jh (s or n) and adds the other half's copy
      const float snd = jh ? s0[q] : s1[q], kp = jh ? s1[q] : s0[q];
      y[q] = kp + __shfl_xor_sync(0xffffffffu, snd, 8);
    }
    const float4 cl = *reinterpret_cast<const float4*>(sm + S::FY + (jh * kK + kk) * kR + i);
    const float4 dl = *reinterpret_cast<const float4*>(sm + S::FY + ((1 - jh) * kK + kk) * kR + i);
    const float4 ex0 = *reinterpret_cast<const float4*>(sm + S::EXY + jh * kR + i);         // Ex[jh][0] at i
    const float4 ex1 = *reinterpret_cast<const float4*>(sm + S::EXY + (2 + jh) * kR + i);   // Ex[jh][1] at i
    const float4 ca = *reinterpret_cast<const float4*>(sm + S::CA + i);
    const float4 cb = *reinterpret_cast<const float4*>(sm + S::CB + i);
    const float4 c1 = *reinterpret_cast<const float4*>(sm + S::CL1 + i);
    const float4 eg = *reinterpret_cast<const float4*>(sm + S::CEG + 4 * k);
    const float ez0 = sm[S::EZ + 4 * k + 2 * jh], ez1 = sm[S::EZ + 4 * k + 2 * jh + 1];   // Ez[0|1][jh] at k
    const float fcy = sm[S::CPS + 8 + jh] + w0 * eg.z, cOy = sm[S::CPS + 2 + jh];
    const float clv[4] = {cl.x, cl.y, cl.z, cl.w}, dlv[4] = {dl.x, dl.y, dl.z, dl.w};
    const float e0v[4] = {ex0.x, ex0.y, ex0.z, ex0.w}, e1v[4] = {ex1.x, ex1.y, ex1.z, ex1.w};
    const float cav[4] = {ca.x, ca.y, ca.z, ca.w}, cbv[4] = {cb.x, cb.y, cb.z, cb.w};
    const float c1v[4] = {c1.x, c1.y, c1.z, c1.w};
    float o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float r = fmaf(w0, c1v[q], fcy) * clv[q];
      r = fmaf(cOy, dlv[q], r);
      r = fmaf(w0, fmaf(cav[q], ez0, fmaf(cbv[q], ez1, fmaf(eg.x, e0v[q], eg.y * e1v[q]))), r);
      o[q] = r - y[q];
      dot = fmaf(clv[q], o[q], dot);
    }
    *reinterpret_cast<float4*>(sm + S::OY + (jh * kK + kk) * kR + i) = make_float4(o[0], o[1], o[2], o[3]);
  }
  __syncthreads();
  // z-face outputs into the (now free) slab area
  store_chunk(sm + S::V, j, c, zb);
  store_chunk(sm + S::V + kZ, j, c, zt);
}

// Scatter-add of one unit's face outputs and the edges and vertices (primary
// part only); returns the edges' and vertices' share of x^T (A x).
__device__ __forceinline__ float slab_scatter(const SemGeom& g, const int* H, int s, int k0, const float* sm,
                                              float* __restrict__ v) {
  using S = SlabSm;
  const int n = g.n, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const float w0 = sm[S::CPS + 32], w02 = sm[S::CPS + 33], d0 = sm[S::CPS + 34];
  const bool lin = lane < n;
  float dot = 0.f;
  // item t = tid + 128 r of each face loop: the lane is the position in the
  // row, the warp and r name the row
  // ---- x- and y-face rows k of the slab: [slot 0..3][kk][lane] of OX, OY
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int slot = r >> 1, kk = w + 4 * (r & 1), k = k0 + kk;
    const int off = H[slot];
    if (off >= 0 && lin && k < n) atomicAdd(v + off + k * n + lane, sm[S::OX + tid + 128 * r]);
  }
  // ---- z-faces, rows j = w + 4 (r & 7)
  const int col0 = (((lane >> 2) ^ (w & 7)) << 2) | (lane & 3);         // swizzled column, rows j = w + 8 t
  const int col1 = (((lane >> 2) ^ ((w + 4) & 7)) << 2) | (lane & 3);   // rows j = w + 4 + 8 t
#pragma unroll 2
  for (int r = 0; r < 16; ++r) {
    const int f = r >> 3, j = w + 4 * (r & 7);
    const int off = H[4 + f];
    if (off >= 0 && j < n && lin) atomicAdd(v + off + j * n + lane, sm[S::V + f * kZ + j * kR + ((r & 1) ? col1 : col0)]);
  }
  // ---- x-edges Ex[sb][sc] at i = l (warp q = sb + 2 sc) and y-edges
  //      Ey[sa][sc] at j = l (q = sa + 2 sc): the line sums along k over the
  //      slab here, the rest of the primary part from slab 0
  {
    const int q = w, l = lane;
    int off = H[6 + q];
    if (off >= 0 && l < n) {
      const int sb = q & 1, sc = q >> 1;
      float sy = 0.f;
#pragma unroll
      for (int kk = 0; kk < kK; ++kk) sy = fmaf(sm[S::CEG + 4 * (k0 + kk) + sc], sm[S::FY + (sb * kK + kk) * kR + l], sy);
      float o = w0 * sy;
      const float exq = sm[S::EXY + q * kR + l];
      if (s == 0) {
        float szc = 0.f;   // sum over j of (c|d)_j F_{4+sc}[j][l] (zero past n)
#pragma unroll
        for (int m = 0; m < kR; ++m) szc = fmaf(sm[S::CCD + 2 * m + sb], sm[S::FZ + sc * kZ + swz(m, l)], szc);
        o = fmaf(w02 * (d0 + sm[S::CL1 + l]) + sm[S::CPS + 12 + q], exq, o);
        o = fmaf(w02, fmaf(sm[S::CA + l], sm[S::VT + 2 * sb + 4 * sc], sm[S::CB + l] * sm[S::VT + 1 + 2 * sb + 4 * sc]), o);
        o = fmaf(w0, szc, o);
        o = fmaf(w0 * sm[S::CPS + 2 + sb], sm[S::EXY + ((1 - sb) + 2 * sc) * kR + l], o);
        o = fmaf(w0 * sm[S::CPS + 4 + sc], sm[S::EXY + (sb + 2 * (1 - sc)) * kR + l], o);
      }
      atomicAdd(v + off + l, o);
      dot = fmaf(exq, o, dot);
    }
    off = H[10 + q];
    if (off >= 0 && l < n) {
      const int sa = q & 1, sc = q >> 1;
      float sx = 0.f;
#pragma unroll
      for (int kk = 0; kk < kK; ++kk) sx = fmaf(sm[S::CEG + 4 * (k0 + kk) + sc], sm[S::FX + (sa * kK + kk) * kR + l], sx);
      float o = w0 * sx;
      const float eyq = sm[S::EXY + (4 + q) * kR + l];
      if (s == 0) {
        float szr = 0.f;   // sum over i of (a|b)_i F_{4+sc}[l][i] (zero past n)
        const float* ab = sm + (sa ? S::CB : S::CA);
        const float* zr = sm + S::FZ + sc * kZ + l * kR;
#pragma unroll
        for (int m4 = 0; m4 < kR / 4; ++m4) {   // chunk m4 of row l sits at chunk m4 ^ (l & 7)
          const float4 zv = *reinterpret_cast<const float4*>(zr + ((m4 ^ (l & 7)) << 2));
          const float4 av = *reinterpret_cast<const float4*>(ab + 4 * m4);
          szr = fmaf(av.x, zv.x, fmaf(av.y, zv.y, fmaf(av.z, zv.z, fmaf(av.w, zv.w, szr))));
        }
        const float2 cd = *reinterpret_cast<const float2*>(sm + S::CCD + 2 * l);
        o = fmaf(w02 * (d0 + sm[S::CL2 + l]) + sm[S::CPS + 16 + q], eyq, o);
        o = fmaf(w02, fmaf(cd.x, sm[S::VT + sa + 4 * sc], cd.y * sm[S::VT + sa + 2 + 4 * sc]), o);
        o = fmaf(w0, szr, o);
        o = fmaf(w0 * sm[S::CPS + sa], sm[S::EXY + (4 + (1 - sa) + 2 * sc) * kR + l], o);
        o = fmaf(w0 * sm[S::CPS + 4 + sc], sm[S::EXY + (4 + sa + 2 * (1 - sc)) * kR + l], o);
      }
      atomicAdd(v + off + l, o);
      dot = fmaf(eyq, o, dot);
    }
  }
  // ---- z-edges Ez[sa][sb] at k in the slab (warp 2: lane = 8 q + kk)
  if (w == 2) {
    const int q = lane >> 3, kk = lane & 7, k = k0 + kk;
    const int off = H[14 + q];
    if (off >= 0 && k < n) {
      const int sa = q & 1, sb = q >> 1;
      const float* ab = sm + (sa ? S::CB : S::CA);
      float syr = 0.f, sxr = 0.f;   // y-face sb row k over i, x-face sa row k over j (zero past n)
#pragma unroll 8
      for (int m = 0; m < kR; ++m) {
        syr = fmaf(ab[m], sm[S::FY + (sb * kK + kk) * kR + m], syr);
        sxr = fmaf(sm[S::CCD + 2 * m + sb], sm[S::FX + (sa * kK + kk) * kR + m], sxr);
      }
      const float4 eg = *reinterpret_cast<const float4*>(sm + S::CEG + 4 * k);
      const float* ez = sm + S::EZ + 4 * k;
      float o = (w02 * (d0 + eg.z) + sm[S::CPS + 20 + q]) * ez[q];
      o = fmaf(w02, fmaf(eg.x, sm[S::VT + sa + 2 * sb], eg.y * sm[S::VT + sa + 2 * sb + 4]), o);
      o = fmaf(w0, syr + sxr, o);
      o = fmaf(w0 * sm[S::CPS + sa], ez[(1 - sa) + 2 * sb], o);
      o = fmaf(w0 * sm[S::CPS + 2 + sb], ez[sa + 2 * (1 - sb)], o);
      atomicAdd(v + off + k, o);
      dot = fmaf(ez[q], o, dot);
    }
  }
  // ---- vertices (slab 0, warp 3)
  if (s == 0 && w == 3 && lane < 8) {
    const int r = lane, sa = r & 1, sb = (r >> 1) & 1, sc = r >> 2;
    const int off = H[18 + r];
    if (off >= 0) {
      const float* ab = sm + (sa ? S::CB : S::CA);
      float sv = 0.f;
#pragma unroll 8
      for (int m = 0; m < kR; ++m) {   // zero past n
        sv = fmaf(ab[m], sm[S::EXY + (sb + 2 * sc) * kR + m], sv);
        sv = fmaf(sm[S::CCD + 2 * m + sb], sm[S::EXY + (4 + sa + 2 * sc) * kR + m], sv);
        sv = fmaf(sm[S::CEG + 4 * m + sc], sm[S::EZ + 4 * m + sa + 2 * sb], sv);
      }
      const float vr = sm[S::VT + r];
      float o = sm[S::CPS + 24 + r] * vr;
      o = fmaf(w02, sv, o);
      o = fmaf(w02 * sm[S::CPS + sa], sm[S::VT + (r ^ 1)], o);
      o = fmaf(w02 * sm[S::CPS + 2 + sb], sm[S::VT + (r ^ 2)], o);
      o = fmaf(w02 * sm[S::CPS + 4 + sc], sm[S::VT + (r ^ 4)], o);
      atomicAdd(v + off, o);
      dot = fmaf(vr, o, dot);
    }
  }
  return dot;
}

__global__ void __launch_bounds__(kSlabThreads, 4)
k_tpt_apply_slab(SemGeom g, SemClassTables<float> tab, const float* __restrict__ u, float* __restrict__ v,
                 double* __restrict__ partials, PcgState* st) {
  extern __shared__ __align__(16) float sm[];
  __shared__ EntityAffine ent[26];
  if (st != nullptr && st->done) return;
  const int tid = threadIdx.x;
  if (tid < 26) entity_affine(g, tid, &ent[tid]);
  const int nslab = (g.n + kK - 1) / kK;
  const long long units = (long long)g.nelem * nslab;
  const long long u_begin = units * blockIdx.x / gridDim.x, u_end = units * (blockIdx.x + 1) / gridDim.x;
  int* H = reinterpret_cast<int*>(sm + SlabSm::HDR);
  float dot = 0.f;
  int e = (int)(u_begin / nslab), s = (int)(u_begin - (long long)e * nslab);   // element and slab of the unit
  for (long long un = u_begin; un < u_end; ++un) {
    const int k0 = s * kK;
    __syncthreads();   // the previous unit is done with the buffers (and ent[] is written)
    if (tid < 27) slab_header(g, tab, ent, e, tid, H);
    __syncthreads();
    slab_gather(g, tab, u, H, k0, sm);
    cp_async_wait<0>();
    __syncthreads();
    slab_faces(g, s, nslab, k0, sm, dot);
    __syncthreads();
    dot += slab_scatter(g, H, s, k0, sm, v);
    if (++s == nslab) {
      s = 0;
      ++e;
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

}  // namespace

void launch_slab_apply(const SemGeom& g, const SemClassTables<float>& t, const float* x, float* y, double* partials,
                       PcgState* st, cudaStream_t s) {
  const size_t smem = (size_t)SlabSm::size * sizeof(float);
  static bool attr = false;
  if (!attr) {   // once; the first launch happens outside any capture
    cudaFuncSetAttribute(k_tpt_apply_slab, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  // one unit per CTA (the block scheduler balances the SMs to within one
  // unit), or contiguous ranges of units once the grid would pass 65536 CTAs
  const long long units = g.nelem * (long long)((g.n + kK - 1) / kK);
  long long grid = units < 65536 ? units : 65536;
  if (grid < 1) grid = 1;
  k_tpt_apply_slab<<<(int)grid, kSlabThreads, smem, s>>>(g, t, x, y, partials, st);
  sem_count_launch();
}

SEM_DEBUG_TU(slab)
