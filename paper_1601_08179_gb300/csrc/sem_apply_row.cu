// Row variant of the transformed condensed operator (Sec. 6, Table 2) for
// FP32 and 2 <= n <= 8: the inner operator of the mixed-precision solve.
//
// The element operator is the one of the other kernels (expansion of the six
// faces into the interior eigenspace, -D^-1, contraction back onto the faces,
// plus the primary part H~_BB on faces, edges and vertices); the mapping of
// the work onto the GPU is built around the skeleton footprint of a row of
// elements along x:
//
// * One CTA takes a segment of up to 32 consecutive elements of one x-row
//   (fixed ey, ez).  Everything such a segment touches in the packed skeleton
//   is 17 contiguous ranges: its x-faces (one range, neighbours share a face),
//   the two y-face and two z-face ranges, four x-edge, two y-edge and two
//   z-edge ranges and four vertex ranges.  The gather is one 1-D bulk copy
//   (cp.async.bulk, completion on an mbarrier) per range into shared memory,
//   the scatter one bulk reduce-add (cp.reduce.async.bulk .add.f32) per range;
//   the at most three unaligned floats at each end of a range go through plain
//   loads and red.global.add.  Entities two elements of the segment share are
//   summed in shared memory first, so they leave the CTA once.
// * Warp w owns the y-plane j = w of the eigenspace cube of every element,
//   lane l owns element l of the segment: the per-plane constants are uniform
//   across a warp and the 1-D basis vectors (K~_{I0}, K~_{Ip}, Lambda) are
//   kernel parameters, so the expansion and contraction factors indexed by i
//   and k are constant-bank operands of the FMAs.
// * Walking k: the x-contraction (over i) and the z-contraction (over k) stay
//   in registers; the y-contraction (over j, i.e. across warps) reads the
//   plane of D^-1 x that every warp stored in shared memory (double buffered,
//   one CTA barrier per k).
// * Face outputs overwrite their inputs in shared memory once no thread reads
//   them any more; edge and vertex outputs are formed first, from the intact
//   inputs, into a separate staging area.

#include <cuda_runtime.h>

#include <cstdint>

#include "sem_device.cuh"
#include "sem_kernels.cuh"

using namespace semdev;

namespace {

constexpr int kRowElems = 32;          // elements per segment (lanes of a warp)
constexpr int kRowBlocks = 17;         // skeleton ranges of a segment
constexpr long long kRowSpin = 1LL << 26;   // bound of the mbarrier wait
// Register cap of the kernel (two CTAs of seven warps share an SM at n = 7; fewer registers spill).
#ifndef SEM_ROW_MAXNREG
#define SEM_ROW_MAXNREG 128
#endif

// 1-D basis of degree p in FP32 (kernel parameter: read through the constant
// bank).  k0 = K~_{I0}, k1 = K~_{Ip}, lam = Lambda, K = K~ corners, w0 = M_00.
struct RowBasis {
  float k0[8], k1[8], lam[8];
  float K[2][2];
  float w0;
};

// Range kinds of a segment, in this order: 0 x-faces, 1-2 y-faces (side sb),
// 3-4 z-faces (side sc), 5-8 x-edges (sb + 2 sc), 9-10 y-edges (sc),
// 11-12 z-edges (sb), 13-16 vertices (sb + 2 sc).
struct RowBlk {
  long long off;   // first float of the range in the skeleton vector
  int len;         // floats
  int head, tail;  // floats [0, head) and [tail, len) by plain accesses, [head, tail) by the bulk engines
  int pad;
};

// Per-segment control, kept in registers: the offset (0..3 floats) of every
// range's first float inside its 16-byte chunk, 2 bits per range (shared
// memory keeps that offset, so the bulk engines see 16-byte aligned middles
// on both sides), and masks of the ranges that lie on the Dirichlet boundary
// entirely, or whose first / last entity does.
struct RowCtl {
  unsigned long long hb;
  unsigned whole, first, last;
  int ex0, Ls, ey, ez;   // the segment: first element, length, row
};

__host__ __device__ constexpr int row_cap(int len) { return (len + 7) & ~3; }
// Largest length of range b for a segment of 32 elements.
__host__ __device__ constexpr int row_len_max(int b, int n) {
  return b == 0 ? (kRowElems + 1) * n * n
                : b <= 4 ? kRowElems * n * n
                         : b <= 8 ? kRowElems * n : b <= 12 ? (kRowElems + 1) * n : kRowElems + 1;
}
// Shared-memory plan: input ranges (faces are overwritten by their outputs),
// output staging for the edge and vertex ranges (5..16), the double-buffered
// planes of D^-1 x ([2][n][n][32]).
template <int N>
struct RowSm {
  static constexpr int cX = row_cap(row_len_max(0, N)), cF = row_cap(row_len_max(1, N));
  static constexpr int cXE = row_cap(row_len_max(5, N)), cE = row_cap(row_len_max(9, N)), cV = row_cap(row_len_max(13, N));
  // first float of input range b (b = 17: end of the input ranges)
  __host__ __device__ static constexpr int base(int b) {
    return b == 0 ? 0
                  : b <= 5 ? cX + (b - 1) * cF
                           : b <= 9 ? cX + 4 * cF + (b - 5) * cXE
                                    : b <= 13 ? cX + 4 * cF + 4 * cXE + (b - 9) * cE
                                              : cX + 4 * cF + 4 * cXE + 4 * cE + (b - 13) * cV;
  }
  // first float of the output staging of range b (5 <= b <= 17)
  __host__ __device__ static constexpr int out_base(int b) {
    return base(kRowBlocks) + (b <= 9 ? (b - 5) * cXE : b <= 13 ? 4 * cXE + (b - 9) * cE : 4 * cXE + 4 * cE + (b - 13) * cV);
  }
  // the same with the range's 16-byte offset: where its first float sits
  __device__ static int start(const RowCtl& c, int b) { return base(b) + (int)((c.hb >> (2 * b)) & 3ull); }
  __device__ static int ostart(const RowCtl& c, int b) {
    return (b <= 4 ? base(b) : out_base(b)) + (int)((c.hb >> (2 * b)) & 3ull);
  }
  static constexpr int BUF = out_base(kRowBlocks);   // one segment's buffer: ranges and output staging
  static constexpr int WB = 2 * BUF;                 // two buffers: the next segment's gather overlaps
  static constexpr int WBS = N * N * kRowElems;      // floats per plane buffer
  static constexpr int total = WB + 2 * WBS;         // floats
  static constexpr size_t bytes = (size_t)total * 4 + 2 * kRowBlocks * sizeof(RowBlk) + 2 * sizeof(RowCtl) + 32;
};

// ---- asynchronous-proxy helpers (mbarrier, bulk copies, bulk reductions) ----
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// global -> shared bulk copy of `bytes` (both addresses 16-byte aligned, bytes
// a multiple of 16), completing on the mbarrier.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// shared -> global element-wise atomic add of `bytes` of floats (same alignment rules).
__device__ __forceinline__ void bulk_reduce_add(float* dst, const void* src, unsigned bytes) {
  asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Waits until the committed bulk operations of this thread have read their shared-memory sources.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Makes this thread's shared-memory writes visible to the asynchronous proxy.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}


// Segment s of an x-row: nseg segments of at most len elements each.
struct RowSeg {
  int nseg, len;
};
inline RowSeg row_segments(int mx) {
  RowSeg r;
  const int nseg0 = (mx + kRowElems - 1) / kRowElems;
  r.len = (mx + nseg0 - 1) / nseg0;           // balanced lengths of at most 32
  r.nseg = (mx + r.len - 1) / r.len;          // so that no segment is empty
  return r;
}

// Skeleton range b of the segment of Ls elements starting at ex0 of row
// (ey, ez): offset, length and Dirichlet flags (layout of sem.h).
__device__ __forceinline__ void row_range(const SemGeom& g, int b, int ex0, int Ls, int ey, int ez, long long* off,
                                          int* len, int* flags) {
  const long long n = g.n, n2 = n * n, mx = g.mx, my = g.my, mz = g.mz;
  const bool first = ex0 == 0, last = ex0 + Ls == g.mx;
  int f = 0;
  if (b == 0) {
    *off = g.off[0] + (ex0 + (mx + 1) * (ey + my * ez)) * n2;
    *len = (Ls + 1) * (int)n2;
    f = (first ? 2 : 0) | (last ? 4 : 0);
  } else if (b <= 2) {
    const long long fy = ey + (b - 1);
    *off = g.off[1] + (ex0 + mx * (fy + (my + 1) * ez)) * n2;
    *len = Ls * (int)n2;
    f = (fy == 0 || fy == my) ? 1 : 0;
  } else if (b <= 4) {
    const long long fz = ez + (b - 3);
    *off = g.off[2] + (ex0 + mx * (ey + my * fz)) * n2;
    *len = Ls * (int)n2;
    f = (fz == 0 || fz == mz) ? 1 : 0;
  } else if (b <= 8) {
    const int q = b - 5;
    const long long vy = ey + (q & 1), vz = ez + (q >> 1);
    *off = g.off[3] + (ex0 + mx * (vy + (my + 1) * vz)) * n;
    *len = Ls * (int)n;
    f = (vy == 0 || vy == my || vz == 0 || vz == mz) ? 1 : 0;
  } else if (b <= 10) {
    const long long vz = ez + (b - 9);
    *off = g.off[4] + (ex0 + (mx + 1) * (ey + my * vz)) * n;
    *len = (Ls + 1) * (int)n;
    f = (vz == 0 || vz == mz) ? 1 : ((first ? 2 : 0) | (last ? 4 : 0));
  } else if (b <= 12) {
    const long long vy = ey + (b - 11);
    *off = g.off[5] + (ex0 + (mx + 1) * (vy + (my + 1) * ez)) * n;
    *len = (Ls + 1) * (int)n;
    f = (vy == 0 || vy == my) ? 1 : ((first ? 2 : 0) | (last ? 4 : 0));
  } else {
    const int q = b - 13;
    const long long vy = ey + (q & 1), vz = ez + (q >> 1);
    *off = g.off[6] + ex0 + (mx + 1) * (vy + (my + 1) * vz);
    *len = Ls + 1;
    f = (vy == 0 || vy == my || vz == 0 || vz == mz) ? 1 : ((first ? 2 : 0) | (last ? 4 : 0));
  }
  *flags = f;
}

// Floats per entity of range b (faces n^2, edges n, vertices 1).
__device__ __forceinline__ int row_entity(int b, int n) { return b <= 4 ? n * n : (b <= 12 ? n : 1); }

// Head and tail of a range for the bulk engines: floats [0, *head) and
// [*tail, len) go through plain accesses, [head, tail) is 16-byte aligned at
// both ends in global memory (and, by construction, in shared memory).
__device__ __forceinline__ void row_split(const float* base, long long off, int len, int* head, int* tail) {
  const unsigned long long lo = (unsigned long long)(base + off), hi = lo + 4ull * (unsigned long long)len;
  const unsigned long long lo16 = (lo + 15ull) & ~15ull, hi16 = hi & ~15ull;
  if (hi16 > lo16) {
    *head = (int)((lo16 - lo) >> 2);
    *tail = (int)((hi16 - lo) >> 2);
  } else {
    *head = len;
    *tail = len;
  }
}

// Describes segment `unit` (warp 0 only, lane b for range b): offsets,
// lengths and aligned middles of its 17 ranges into blk, the control word into
// *ctl.  Shared memory keeps each range's global address modulo 16 bytes
// (input and output vectors agree on it).
template <int N>
__device__ __forceinline__ void row_describe(const SemGeom& g, const RowSeg& seg, long long unit, const float* v,
                                             RowBlk* blk, RowCtl* ctl) {
  const int b = threadIdx.x;
  const int sg = (int)(unit % seg.nseg);
  const long long r = unit / seg.nseg;
  const int ey = (int)(r % g.my), ez = (int)(r / g.my);
  const int ex0 = sg * seg.len;
  const int Ls = min(seg.len, g.mx - ex0);
  long long off = 0;
  int len = 0, flags = 1, h = 0;
  if (b < kRowBlocks) {
    row_range(g, b, ex0, Ls, ey, ez, &off, &len, &flags);
#ifdef SEM_DEBUG
    // a range reaching past the checked bound is recorded and skipped (treated as Dirichlet)
    if (!(flags & 1) && !sem_dbg_ok(off, len, g.dbg_bound)) flags = 1;
#endif
    h = (int)(((unsigned long long)(v + off) >> 2) & 3ull);
    RowBlk d;
    d.off = off;
    d.len = len;
    row_split(v, off, len, &d.head, &d.tail);
    d.pad = 0;
    blk[b] = d;
  }
  const unsigned h0 = __ballot_sync(0xffffffffu, h & 1), h1 = __ballot_sync(0xffffffffu, (h >> 1) & 1);
  const unsigned wh = __ballot_sync(0xffffffffu, b < kRowBlocks && (flags & 1));
  const unsigned fi = __ballot_sync(0xffffffffu, b < kRowBlocks && (flags & 2));
  const unsigned la = __ballot_sync(0xffffffffu, b < kRowBlocks && (flags & 4));
  if (b == 0) {
    unsigned long long hb = 0;
    for (int q = 0; q < kRowBlocks; ++q)
      hb |= (unsigned long long)(((h0 >> q) & 1u) | (((h1 >> q) & 1u) << 1)) << (2 * q);
    RowCtl cc;
    cc.hb = hb;
    cc.whole = wh;
    cc.first = fi;
    cc.last = la;
    cc.ex0 = ex0;
    cc.Ls = Ls;
    cc.ey = ey;
    cc.ez = ez;
    *ctl = cc;
  }
  __syncwarp();
}

// Gather of a described segment into one buffer (warp 0 only): lane b issues
// the bulk copy of range b's aligned middle (all completing on `bar`), then
// the lanes load the unaligned ends and zero the ranges on the Dirichlet
// boundary.
template <int N>
__device__ __forceinline__ void row_prefetch(const float* __restrict__ u, float* S, const RowBlk* blk, const RowCtl& c,
                                             unsigned long long* bar) {
  using Sm = RowSm<N>;
  const int lane = threadIdx.x;
  const bool mine = lane < kRowBlocks && !((c.whole >> lane) & 1u);
  const unsigned bytes = mine ? 4u * (unsigned)(blk[lane].tail - blk[lane].head) : 0u;
  unsigned total = bytes;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
  if (lane == 0) mbar_arrive_expect_tx(bar, total);
  __syncwarp();
  if (bytes != 0u) bulk_load(S + Sm::start(c, lane) + blk[lane].head, u + blk[lane].off + blk[lane].head, bytes, bar);
  for (int idx = lane; idx < kRowBlocks * 8; idx += 32) {
    const int b = idx >> 3, e = idx & 7;
    if ((c.whole >> b) & 1u) continue;
    const int pos = e < 4 ? e : blk[b].tail + (e - 4);
    if (e < 4 ? pos < blk[b].head : pos < blk[b].len) S[Sm::start(c, b) + pos] = u[blk[b].off + pos];
  }
  for (unsigned m = c.whole; m != 0u; m &= m - 1u) {
    const int b = __ffs(m) - 1, st = Sm::start(c, b), len = blk[b].len;
    for (int t = lane; t < len; t += 32) S[st + t] = 0.f;
  }
}

// Bounded wait for the bulk copies of one buffer (phase `parity` of its barrier).
__device__ __forceinline__ bool row_wait(unsigned long long* bar, unsigned parity) {
  long long spins = 0;
  bool done = mbar_try_wait(bar, parity);
  while (!done && ++spins < kRowSpin) done = mbar_try_wait(bar, parity);
  return done;
}

// Zeros the first / last entity of the ranges that start or end on the
// Dirichlet boundary (x = 0 or x = 1), at the input (out = false) or output
// positions.
template <int N>
__device__ __forceinline__ void row_zero_ends(float* S, const RowBlk* blk, const RowCtl& c, bool out) {
  using Sm = RowSm<N>;
  for (unsigned m = (c.first | c.last) & ~c.whole; m != 0u; m &= m - 1u) {
    const int b = __ffs(m) - 1;
    const int es = row_entity(b, N), st = out ? Sm::ostart(c, b) : Sm::start(c, b), len = blk[b].len;
    for (int t = threadIdx.x; t < es; t += blockDim.x) {
      if ((c.first >> b) & 1u) S[st + t] = 0.f;
      if ((c.last >> b) & 1u) S[st + len - es + t] = 0.f;
    }
  }
}

// Scatter-add of a segment's outputs: lane b of warp 0 issues the bulk
// reduce-add of range b's aligned middle and commits it (not waited for
// here), every thread takes part in the red.global.add of the ends; ranges on
// the Dirichlet boundary are skipped.  The caller has fenced its
// shared-memory writes for the asynchronous proxy and synchronised the CTA.
template <int N>
__device__ __forceinline__ void row_scatter(float* __restrict__ v, const float* S, const RowBlk* blk, const RowCtl& c) {
  using Sm = RowSm<N>;
  if (threadIdx.x < kRowBlocks && !((c.whole >> threadIdx.x) & 1u)) {
    const int b = threadIdx.x;
    const int h = blk[b].head, t = blk[b].tail;
    if (t > h) bulk_reduce_add(v + blk[b].off + h, S + Sm::ostart(c, b) + h, 4u * (unsigned)(t - h));
  }
  if (threadIdx.x < 32) bulk_commit();
  for (int idx = threadIdx.x; idx < kRowBlocks * 8; idx += blockDim.x) {
    const int b = idx >> 3, e = idx & 7;
    if ((c.whole >> b) & 1u) continue;
    const int pos = e < 4 ? e : blk[b].tail + (e - 4);
    if (e < 4 ? pos < blk[b].head : pos < blk[b].len) red_add(v + blk[b].off + pos, S[Sm::ostart(c, b) + pos]);
  }
}

// Primary part of the 12 edges of element `el` at position p = warp index
// (one value per edge), and of its vertices (warp w takes the vertex pairs
// (sb, sc) = w, w + N, ...), from the intact inputs; outputs into the staging
// area, the entities shared with the x-neighbour added in two steps.  Also
// returns the edge values at p (x-edges exv[sb + 2 sc], y-edges
// eyv[sa + 2 sc]) that the face outputs need.  Returns this thread's share of
// u^T (A u).
template <int N>
__device__ __forceinline__ float row_edges(float* S, const RowCtl& c, const RowBasis& bf, const RowBasis& sbf,
                                           float d0, float d1, float d2, float d3, int el, int Ls, float (&exv)[4],
                                           float (&eyv)[4]) {
  using Sm = RowSm<N>;
  constexpr int n2 = N * N;
  const int lane = threadIdx.x & 31, p = threadIdx.x >> 5;
  const bool act = lane < Ls, next = lane + 1 < Ls;
  const float w0 = bf.w0, w02 = w0 * w0;
  const float k0p = sbf.k0[p], k1p = sbf.k1[p], lamp = sbf.lam[p];   // runtime index: the shared copy
  // line sums of the six faces through position p: columns (index p of the
  // fast coordinate, summed over the slow one) and rows (the reverse), with
  // the factors K~_{I0} (s = 0) and K~_{Ip} (s = 1):  c?[2 side + s], r?[2 side + s]
  float zc[4] = {0.f, 0.f, 0.f, 0.f}, zr[4] = {0.f, 0.f, 0.f, 0.f};
  float yc[4] = {0.f, 0.f, 0.f, 0.f}, yr[4] = {0.f, 0.f, 0.f, 0.f};
  float xc[4] = {0.f, 0.f, 0.f, 0.f}, xr[4] = {0.f, 0.f, 0.f, 0.f};
  {
    const float* x0 = S + Sm::start(c, 0) + el * n2;
    const float* x1 = x0 + n2;
    const float* y0 = S + Sm::start(c, 1) + el * n2;
    const float* y1 = S + Sm::start(c, 2) + el * n2;
    const float* z0 = S + Sm::start(c, 3) + el * n2;
    const float* z1 = S + Sm::start(c, 4) + el * n2;
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const float a0 = bf.k0[m], a1 = bf.k1[m];
      float t;
      t = z0[m * N + p]; zc[0] = fmaf(a0, t, zc[0]); zc[1] = fmaf(a1, t, zc[1]);
      t = z1[m * N + p]; zc[2] = fmaf(a0, t, zc[2]); zc[3] = fmaf(a1, t, zc[3]);
      t = z0[p * N + m]; zr[0] = fmaf(a0, t, zr[0]); zr[1] = fmaf(a1, t, zr[1]);
      t = z1[p * N + m]; zr[2] = fmaf(a0, t, zr[2]); zr[3] = fmaf(a1, t, zr[3]);
      t = y0[m * N + p]; yc[0] = fmaf(a0, t, yc[0]); yc[1] = fmaf(a1, t, yc[1]);
      t = y1[m * N + p]; yc[2] = fmaf(a0, t, yc[2]); yc[3] = fmaf(a1, t, yc[3]);
      t = y0[p * N + m]; yr[0] = fmaf(a0, t, yr[0]); yr[1] = fmaf(a1, t, yr[1]);
      t = y1[p * N + m]; yr[2] = fmaf(a0, t, yr[2]); yr[3] = fmaf(a1, t, yr[3]);
      t = x0[m * N + p]; xc[0] = fmaf(a0, t, xc[0]); xc[1] = fmaf(a1, t, xc[1]);
      t = x1[m * N + p]; xc[2] = fmaf(a0, t, xc[2]); xc[3] = fmaf(a1, t, xc[3]);
      t = x0[p * N + m]; xr[0] = fmaf(a0, t, xr[0]); xr[1] = fmaf(a1, t, xr[1]);
      t = x1[p * N + m]; xr[2] = fmaf(a0, t, xr[2]); xr[3] = fmaf(a1, t, xr[3]);
    }
  }
  float ezv[4], V[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int s1 = q & 1, s2 = q >> 1;
    exv[q] = S[Sm::start(c, 5 + q) + el * N + p];                 // Ex[sb = s1][sc = s2] at i = p
    eyv[q] = S[Sm::start(c, 9 + s2) + (el + s1) * N + p];         // Ey[sa = s1][sc = s2] at j = p
    ezv[q] = S[Sm::start(c, 11 + s2) + (el + s1) * N + p];        // Ez[sa = s1][sb = s2] at k = p
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) V[r] = S[Sm::start(c, 13 + ((r >> 1) & 1) + 2 * (r >> 2)) + el + (r & 1)];
  float dot = 0.f;
  // x-edges Ex[sb][sc] at i = p: not shared inside the segment
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int sb = q & 1, sc = q >> 1;
    float o = (w02 * fmaf(d1, lamp, d0) + w0 * (d2 * bf.K[sb][sb] + d3 * bf.K[sc][sc])) * exv[q];
    o = fmaf(w02 * d1, fmaf(k0p, V[2 * sb + 4 * sc], k1p * V[1 + 2 * sb + 4 * sc]), o);
    o = fmaf(w0, fmaf(d2, zc[2 * sc + sb], d3 * yc[2 * sb + sc]), o);
    o = fmaf(w0 * d2 * bf.K[sb][1 - sb], exv[(1 - sb) + 2 * sc], o);
    o = fmaf(w0 * d3 * bf.K[sc][1 - sc], exv[sb + 2 * (1 - sc)], o);
    if (act) {
      S[Sm::ostart(c, 5 + q) + el * N + p] = o;
      dot = fmaf(exv[q], o, dot);
    }
  }
  // y-edges Ey[sa][sc] at j = p and z-edges Ez[sa][sb] at k = p: the sa = 1
  // entity of element l is the sa = 0 entity of element l + 1
  float oy[4], oz[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int sa = q & 1, s2 = q >> 1;
    {   // y-edge, sc = s2
      const int sc = s2;
      float o = (w02 * fmaf(d2, lamp, d0) + w0 * (d1 * bf.K[sa][sa] + d3 * bf.K[sc][sc])) * eyv[q];
      o = fmaf(w02 * d2, fmaf(k0p, V[sa + 4 * sc], k1p * V[sa + 2 + 4 * sc]), o);
      o = fmaf(w0, fmaf(d1, zr[2 * sc + sa], d3 * xc[2 * sa + sc]), o);
      o = fmaf(w0 * d1 * bf.K[sa][1 - sa], eyv[(1 - sa) + 2 * sc], o);
      o = fmaf(w0 * d3 * bf.K[sc][1 - sc], eyv[sa + 2 * (1 - sc)], o);
      oy[q] = o;
    }
    {   // z-edge, sb = s2
      const int sb = s2;
      float o = (w02 * fmaf(d3, lamp, d0) + w0 * (d1 * bf.K[sa][sa] + d2 * bf.K[sb][sb])) * ezv[q];
      o = fmaf(w02 * d3, fmaf(k0p, V[sa + 2 * sb], k1p * V[sa + 2 * sb + 4]), o);
      o = fmaf(w0, fmaf(d1, yr[2 * sb + sa], d2 * xr[2 * sa + sb]), o);
      o = fmaf(w0 * d1 * bf.K[sa][1 - sa], ezv[(1 - sa) + 2 * sb], o);
      o = fmaf(w0 * d2 * bf.K[sb][1 - sb], ezv[sa + 2 * (1 - sb)], o);
      oz[q] = o;
    }
    if (act) dot = fmaf(eyv[q], oy[q], fmaf(ezv[q], oz[q], dot));
  }
#pragma unroll
  for (int s2 = 0; s2 < 2; ++s2) {
    if (act) {
      S[Sm::ostart(c, 9 + s2) + el * N + p] = oy[2 * s2];
      S[Sm::ostart(c, 11 + s2) + el * N + p] = oz[2 * s2];
    }
  }
  __syncwarp();
#pragma unroll
  for (int s2 = 0; s2 < 2; ++s2) {
    if (act) {
      float* ty = S + Sm::ostart(c, 9 + s2) + (el + 1) * N + p;
      float* tz = S + Sm::ostart(c, 11 + s2) + (el + 1) * N + p;
      *ty = next ? *ty + oy[1 + 2 * s2] : oy[1 + 2 * s2];
      *tz = next ? *tz + oz[1 + 2 * s2] : oz[1 + 2 * s2];
    }
  }
  // vertices (sa, sb, sc), r = sa + 2 sb + 4 sc
  for (int pr = p; pr < 4; pr += N) {
    const int sb = pr & 1, sc = pr >> 1;
    const float* xe = S + Sm::start(c, 5 + sb + 2 * sc) + el * N;
    const float* vt = S + Sm::start(c, 13 + pr) + el;
    float ov[2];
#pragma unroll
    for (int sa = 0; sa < 2; ++sa) {
      const float* ye = S + Sm::start(c, 9 + sc) + (el + sa) * N;
      const float* ze = S + Sm::start(c, 11 + sb) + (el + sa) * N;
      float ls = 0.f;
#pragma unroll
      for (int m = 0; m < N; ++m) {
        const float ka = sa ? bf.k1[m] : bf.k0[m];
        const float kb = sb ? bf.k1[m] : bf.k0[m];   // selects between two constant operands
        const float kc = sc ? bf.k1[m] : bf.k0[m];
        ls = fmaf(d1 * ka, xe[m], fmaf(d2 * kb, ye[m], fmaf(d3 * kc, ze[m], ls)));
      }
      const float vr = vt[sa];
      const float vd = w0 * w02 * d0 + w02 * (d1 * bf.K[sa][sa] + d2 * sbf.K[sb][sb] + d3 * sbf.K[sc][sc]);
      float o = fmaf(vd, vr, w02 * ls);
      o = fmaf(w02 * d1 * bf.K[sa][1 - sa], vt[1 - sa], o);                                  // r ^ 1
      o = fmaf(w02 * d2 * sbf.K[sb][1 - sb], S[Sm::start(c, 13 + (pr ^ 1)) + el + sa], o);     // r ^ 2
      o = fmaf(w02 * d3 * sbf.K[sc][1 - sc], S[Sm::start(c, 13 + (pr ^ 2)) + el + sa], o);     // r ^ 4
      ov[sa] = o;
      if (act) dot = fmaf(vr, o, dot);
    }
    if (act) S[Sm::ostart(c, 13 + pr) + el] = ov[0];
    __syncwarp();
    if (act) {
      float* t = S + Sm::ostart(c, 13 + pr) + el + 1;
      *t = next ? *t + ov[1] : ov[1];
    }
  }
  return dot;
}

// The element operator of one described, gathered segment (buffer S):
// edges and vertices, the walk over k, the z-faces; outputs in the buffer.
// Returns this thread's share of u^T (A u).
template <int N>
__device__ __forceinline__ float row_compute(const SemGeom& g, const SemClassTables<float>& tab, const RowBasis& bf,
                                             const RowBasis& sbf, float* S, float* WB, const RowCtl& c) {
  using Sm = RowSm<N>;
  constexpr int n2 = N * N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // element constants: metric coefficients d of the element's width class
  const bool act = lane < c.Ls;
  const int el = act ? lane : 0;
  const int cls = elem_class(g, tab, c.ex0 + el, c.ey, c.ez);
  const float4 dd = __ldg(reinterpret_cast<const float4*>(tab.dcoef) + cls);
  const float d0 = dd.x, d1 = dd.y, d2 = dd.z, d3 = dd.w;
  const float w0 = bf.w0;

  float exv[4], eyv[4];
  float dot = row_edges<N>(S, c, bf, sbf, d0, d1, d2, d3, el, c.Ls, exv, eyv);
  __syncthreads();   // every line sum is taken before the faces are overwritten

  // ---- walk the y-plane j = w in k
  const int j = w;
  const float k0j = sbf.k0[j], k1j = sbf.k1[j], lamj = sbf.lam[j];
  const float cj = d2 * k0j, dj = d2 * k1j, ai = d1 * k0j, bi = d1 * k1j;
  const float sj = fmaf(d2, lamj, d0);          // D_ijk = sj + d1 lam_i + d3 lam_k
  const float l1w = d1 * lamj, l2w = d2 * lamj;
  float* XF = S + Sm::start(c, 0);
  float* YF0 = S + Sm::start(c, 1);
  float* YF1 = S + Sm::start(c, 2);
  const float* ZE0 = S + Sm::start(c, 11);
  const float* ZE1 = S + Sm::start(c, 12);
  float e4h[N], e5h[N], z4[N], z5[N];
  {
    const float* z0 = S + Sm::start(c, 3) + el * n2 + j * N;
    const float* z1 = S + Sm::start(c, 4) + el * n2 + j * N;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      e4h[i] = d3 * z0[i];
      e5h[i] = d3 * z1[i];
      z4[i] = 0.f;
      z5[i] = 0.f;
    }
  }
  const float fx0 = fmaf(d0, w0, d1 * bf.K[0][0]), fx1 = fmaf(d0, w0, d1 * bf.K[1][1]);
  const float cx0 = d1 * bf.K[0][1], cx1 = d1 * bf.K[1][0];
  const float fy0 = fmaf(d0, w0, d2 * bf.K[0][0]), fy1 = fmaf(d0, w0, d2 * bf.K[1][1]);
  const float cy0 = d2 * bf.K[0][1], cy1 = d2 * bf.K[1][0];
  const int xo = el * n2 + j;        // x-face (k, j) of element el: xo + k N
  const int yo = el * n2 + w;        // y-face (k, i = w): yo + k N
#pragma unroll 1
  for (int k = 0; k < N; ++k) {   // not unrolled: registers for occupancy; the k factors come from shared memory
    const float k0k = sbf.k0[k], k1k = sbf.k1[k], lamk = sbf.lam[k];
    const float A = XF[xo + k * N], B = XF[xo + n2 + k * N];
    float C[N], D[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      C[i] = YF0[el * n2 + k * N + i];
      D[i] = YF1[el * n2 + k * N + i];
    }
    float ezk[4];   // Ez[sa][sb] at k, index sa + 2 sb
    ezk[0] = ZE0[el * N + k];
    ezk[1] = ZE0[(el + 1) * N + k];
    ezk[2] = ZE1[el * N + k];
    ezk[3] = ZE1[(el + 1) * N + k];
    const float Ah = d1 * A, Bh = d1 * B, denb = fmaf(d3, lamk, sj);
    float sx0 = 0.f, sx1 = 0.f;
    float* wb = WB + (k & 1) * Sm::WBS + j * N * 32 + lane;   // planes [j][i][lane]
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float x = bf.k0[i] * Ah;
      x = fmaf(bf.k1[i], Bh, x);
      x = fmaf(cj, C[i], x);
      x = fmaf(dj, D[i], x);
      x = fmaf(k0k, e4h[i], x);
      x = fmaf(k1k, e5h[i], x);
      const float wv = x * rcp_approx(fmaf(d1, bf.lam[i], denb));   // D^-1 x (sign at the outputs)
      sx0 = fmaf(bf.k0[i], wv, sx0);
      sx1 = fmaf(bf.k1[i], wv, sx1);
      z4[i] = fmaf(k0k, wv, z4[i]);
      z5[i] = fmaf(k1k, wv, z5[i]);
      wb[i * 32] = wv;
    }
    // x-faces at (k, j): diagonal, opposite face, the four edge lines, -condensed
    const float ek = d3 * k0k, gk = d3 * k1k;
    const float bx = w0 * fmaf(d3, lamk, l2w);
    float o0 = (fx0 + bx) * A;
    o0 = fmaf(cx0, B, o0);
    o0 = fmaf(w0, fmaf(cj, ezk[0], fmaf(dj, ezk[2], fmaf(ek, eyv[0], gk * eyv[2]))), o0);
    o0 = fmaf(-d1, sx0, o0);
    float o1 = (fx1 + bx) * B;
    o1 = fmaf(cx1, A, o1);
    o1 = fmaf(w0, fmaf(cj, ezk[1], fmaf(dj, ezk[3], fmaf(ek, eyv[1], gk * eyv[3]))), o1);
    o1 = fmaf(-d1, sx1, o1);
    if (act) dot = fmaf(A, o0, fmaf(B, o1, dot));
    __syncwarp();
    if (act) XF[xo + k * N] = o0;
    __syncwarp();
    if (act) {
      float* t = XF + xo + n2 + k * N;
      *t = lane + 1 < c.Ls ? *t + o1 : o1;
    }
    __syncthreads();   // the plane k of D^-1 x is complete; every row k of the y-faces has been read
    // y-faces at (k, i = w): sums over the planes j of D^-1 x
    const float Cv = YF0[yo + k * N], Dv = YF1[yo + k * N];
    const float* wr = WB + (k & 1) * Sm::WBS + w * 32 + lane;
    float y0 = 0.f, y1 = 0.f;
#pragma unroll
    for (int jj = 0; jj < N; ++jj) {
      const float t = wr[jj * N * 32];
      y0 = fmaf(bf.k0[jj], t, y0);
      y1 = fmaf(bf.k1[jj], t, y1);
    }
    const float by = w0 * fmaf(d3, lamk, l1w);
    float o2 = (fy0 + by) * Cv;
    o2 = fmaf(cy0, Dv, o2);
    o2 = fmaf(w0, fmaf(ai, ezk[0], fmaf(bi, ezk[1], fmaf(ek, exv[0], gk * exv[2]))), o2);
    o2 = fmaf(-d2, y0, o2);
    float o3 = (fy1 + by) * Dv;
    o3 = fmaf(cy1, Cv, o3);
    o3 = fmaf(w0, fmaf(ai, ezk[2], fmaf(bi, ezk[3], fmaf(ek, exv[1], gk * exv[3]))), o3);
    o3 = fmaf(-d2, y1, o3);
    if (act) {
      dot = fmaf(Cv, o2, fmaf(Dv, o3, dot));
      YF0[yo + k * N] = o2;
      YF1[yo + k * N] = o3;
    }
  }

  // ---- z-faces at (j, i): row j of each, from the z-sums of the k walk
  {
    const float fz0 = fmaf(d0, w0, d3 * bf.K[0][0]), fz1 = fmaf(d0, w0, d3 * bf.K[1][1]);
    const float cz0 = d3 * bf.K[0][1], cz1 = d3 * bf.K[1][0];
    float* z0 = S + Sm::start(c, 3) + el * n2 + j * N;
    float* z1 = S + Sm::start(c, 4) + el * n2 + j * N;
    const float* xe0 = S + Sm::start(c, 5) + el * N;   // Ex[sb][sc], slot sb + 2 sc
    const float* xe1 = S + Sm::start(c, 6) + el * N;
    const float* xe2 = S + Sm::start(c, 7) + el * N;
    const float* xe3 = S + Sm::start(c, 8) + el * N;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float E4 = z0[i], E5 = z1[i];
      const float a_i = d1 * bf.k0[i], b_i = d1 * bf.k1[i];
      const float bz = w0 * fmaf(d1, bf.lam[i], l2w);
      float o4 = (fz0 + bz) * E4;
      o4 = fmaf(cz0, E5, o4);
      o4 = fmaf(w0, fmaf(a_i, eyv[0], fmaf(b_i, eyv[1], fmaf(cj, xe0[i], dj * xe1[i]))), o4);
      o4 = fmaf(-d3, z4[i], o4);
      float o5 = (fz1 + bz) * E5;
      o5 = fmaf(cz1, E4, o5);
      o5 = fmaf(w0, fmaf(a_i, eyv[2], fmaf(b_i, eyv[3], fmaf(cj, xe2[i], dj * xe3[i]))), o5);
      o5 = fmaf(-d3, z5[i], o5);
      if (act) {
        dot = fmaf(E4, o4, fmaf(E5, o5, dot));
        z0[i] = o4;
        z1[i] = o5;
      }
    }
  }
  return dot;
}

// v += Hhat~ u, one x-row segment at a time per CTA (a persistent grid: while
// a segment is computed, the next one's ranges are on their way into the
// other buffer); returns, when st is given, p^T A p and alpha as the other
// operator kernels do.
template <int N>
__global__ void __maxnreg__(SEM_ROW_MAXNREG)
k_tpt_apply_row(SemGeom g, SemClassTables<float> tab, RowBasis bf, RowSeg seg, const float* __restrict__ u,
                float* __restrict__ v, double* __restrict__ partials, PcgState* st) {
  using Sm = RowSm<N>;
  extern __shared__ __align__(16) float S[];
  RowBlk* blk = reinterpret_cast<RowBlk*>(S + Sm::total);                  // [2][17]
  RowCtl* ctl = reinterpret_cast<RowCtl*>(blk + 2 * kRowBlocks);           // [2]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(ctl + 2);   // [2]
  __shared__ RowBasis sbf;   // for indices known at run time only (a kernel parameter indexed so would go to the stack)
  if (st != nullptr && st->done) return;
  const long long units = (long long)seg.nseg * g.my * g.mz;
  const bool warp0 = threadIdx.x < 32;
  if (threadIdx.x == 0) {
    sbf = bf;
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp0 && (long long)blockIdx.x < units) {
    row_describe<N>(g, seg, blockIdx.x, v, blk, ctl);
    row_prefetch<N>(u, S, blk, ctl[0], bar);
  }
  __syncthreads();
  float dot = 0.f;
  unsigned phase = 0u;   // bit b: parity of the next completion of bar[b]
  int t = 0;
  bool failed = false;
  for (long long un = blockIdx.x; un < units; un += gridDim.x, ++t) {
    const int b = t & 1;
    float* Sb = S + b * Sm::BUF;
    // the next segment into the other buffer, once the previous scatter from it has read its sources
    const long long nx = un + gridDim.x;
    if (warp0) {
      bulk_wait_read();
      __syncwarp();
      if (nx < units) {
        row_describe<N>(g, seg, nx, v, blk + (b ^ 1) * kRowBlocks, ctl + (b ^ 1));
        row_prefetch<N>(u, S + (b ^ 1) * Sm::BUF, blk + (b ^ 1) * kRowBlocks, ctl[b ^ 1], bar + (b ^ 1));
      }
    }
    const RowCtl c = ctl[b];
    const RowBlk* bk = blk + b * kRowBlocks;
    const bool ok = row_wait(bar + b, (phase >> b) & 1u);
    phase ^= 1u << b;
    if (__syncthreads_or(!ok)) {   // the copies did not complete in time: stop the solve
      failed = true;
      break;
    }
    row_zero_ends<N>(Sb, bk, c, false);
    __syncthreads();
    dot += row_compute<N>(g, tab, bf, sbf, Sb, S + Sm::WB, c);
    __syncthreads();
    row_zero_ends<N>(Sb, bk, c, true);
    fence_async_smem();
    __syncthreads();
    row_scatter<N>(v, Sb, bk, c);
    __syncthreads();   // the ends are read before the next gather into this buffer writes them
  }
  if (warp0) bulk_wait_all();
  if (failed) {
    if (threadIdx.x == 0 && st != nullptr) st->done = 2;
    return;
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

RowBasis row_basis(const SemBasis& b) {
  RowBasis r{};
  for (int i = 0; i < b.n && i < 8; ++i) {
    r.k0[i] = (float)b.k[0][i];
    r.k1[i] = (float)b.k[1][i];
    r.lam[i] = (float)b.lam[i];
  }
  for (int s = 0; s < 2; ++s)
    for (int t = 0; t < 2; ++t) r.K[s][t] = (float)b.K[s][t];
  r.w0 = (float)b.w0;
  return r;
}

template <int N>
void launch_row_n(const SemGeom& g, const SemBasis& b, const SemClassTables<float>& t, const float* x, float* y,
                  double* partials, PcgState* st, cudaStream_t s) {
  static int resident = 0;
  if (resident == 0) {   // once per instantiation; the first launch happens outside any capture
    cudaFuncSetAttribute(k_tpt_apply_row<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RowSm<N>::bytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_tpt_apply_row<N>, N * 32, RowSm<N>::bytes);
    if (resident < 1) resident = 1;
  }
  const RowSeg seg = row_segments(g.mx);
  const long long units = (long long)seg.nseg * g.my * g.mz;
  // a persistent grid: every resident CTA walks segments blockIdx.x, + gridDim.x, ...
  long long grid = (long long)sem_num_sms() * resident;
  if (grid > units) grid = units;
  k_tpt_apply_row<N><<<(unsigned)grid, N * 32, RowSm<N>::bytes, s>>>(g, t, row_basis(b), seg, x, y, partials, st);
  sem_count_launch();
}

}  // namespace

bool row_usable(const SemGeom& g, const float* x, const float* y) {
  if (!row_supported(g.n)) return false;
  const RowSeg seg = row_segments(g.mx);
  const long long units = (long long)seg.nseg * g.my * g.mz;
  // the bulk engines need input and output at the same address modulo 16 bytes
  const bool same_mod16 = ((reinterpret_cast<uintptr_t>(x) ^ reinterpret_cast<uintptr_t>(y)) & 15u) == 0;
  return units <= kRowMaxUnits && same_mod16;
}

void launch_row_apply(const SemGeom& g, const SemBasis& b, const SemClassTables<float>& t, const float* x, float* y,
                      double* partials, PcgState* st, cudaStream_t s) {
  switch (g.n) {
    case 2: launch_row_n<2>(g, b, t, x, y, partials, st, s); return;
    case 3: launch_row_n<3>(g, b, t, x, y, partials, st, s); return;
    case 4: launch_row_n<4>(g, b, t, x, y, partials, st, s); return;
    case 5: launch_row_n<5>(g, b, t, x, y, partials, st, s); return;
    case 6: launch_row_n<6>(g, b, t, x, y, partials, st, s); return;
    case 7: launch_row_n<7>(g, b, t, x, y, partials, st, s); return;
    default: launch_row_n<8>(g, b, t, x, y, partials, st, s); return;
  }
}

SEM_DEBUG_TU(row)
