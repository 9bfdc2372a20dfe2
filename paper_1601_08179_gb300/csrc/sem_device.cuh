// Device helpers shared by the kernels of the condensed spectral-element library.
#pragma once

#include <cuda_runtime.h>

#include "sem_internal.h"

namespace semdev {

// ---------------------------------------------------------------------------
// Debug builds (-DSEM_DEBUG): bounds record of the entity offsets
// ---------------------------------------------------------------------------
// Every skeleton access of a kernel is an entity offset (formed by
// face_base / edge_base / vert_index or entity_offset below) plus a local
// index that the loops keep inside the entity (n^2 values of a face, n of an
// edge, one vertex).  A debug build checks each offset it forms, and each class
// index, against its range before any access; a failing one is counted, the
// first offending value kept, and the entity treated as absent (no gather, no
// scatter), so the kernel goes on without touching memory out of range.
// Release builds compile every check to nothing.  The record is per
// translation unit; SEM_DEBUG_TU defines its host reader.
#ifdef SEM_DEBUG
static __device__ unsigned long long sem_dbg_count;
static __device__ long long sem_dbg_first;

static __device__ __forceinline__ bool sem_dbg_ok(long long v, long long extent, long long bound) {
  if (v >= 0 && v + extent <= bound) return true;
  if (atomicAdd(&sem_dbg_count, 1ull) == 0ull) sem_dbg_first = v;
  return false;
}
#endif

// An entity offset `off` of `extent` values, formed by a kernel: returned as is
// in release builds; in debug builds a non-Dirichlet offset reaching past the
// checked bound (N_B, unless lowered by sem_debug_limit_skeleton) is recorded
// and turned into "Dirichlet" (*dir = true).
static __device__ __forceinline__ long long sem_dbg_entity(long long off, long long extent, const SemGeom& g,
                                                           bool* dir) {
#ifdef SEM_DEBUG
  if (!*dir && !sem_dbg_ok(off, extent, g.dbg_bound)) *dir = true;
#else
  (void)extent; (void)g; (void)dir;
#endif
  return off;
}

// ---------------------------------------------------------------------------
// Mesh helpers
// ---------------------------------------------------------------------------
static __device__ __forceinline__ void elem_coords(const SemGeom& g, long long e, int* ex, int* ey, int* ez) {
  *ex = (int)(e % g.mx);
  long long r = e / g.mx;
  *ey = (int)(r % g.my);
  *ez = (int)(r / g.my);
}

// Element visiting order of the operator kernels: the axis with the most width
// classes is slowest, so consecutive elements share their class tables.
static __device__ __forceinline__ void elem_visit(const SemGeom& g, long long e, int* ex, int* ey, int* ez) {
  if (g.slow == 0) {
    const long long r = e % ((long long)g.my * g.mz);
    *ex = (int)(e / ((long long)g.my * g.mz));
    *ey = (int)(r % g.my);
    *ez = (int)(r / g.my);
  } else if (g.slow == 1) {
    const long long r = e % ((long long)g.mx * g.mz);
    *ey = (int)(e / ((long long)g.mx * g.mz));
    *ex = (int)(r % g.mx);
    *ez = (int)(r / g.mx);
  } else {
    elem_coords(g, e, ex, ey, ez);
  }
}

// Face slot 0..5 = (dir, side): 0 w, 1 e, 2 s, 3 n, 4 b, 5 t.
static __device__ __forceinline__ long long face_base(const SemGeom& g, int ex, int ey, int ez, int slot, bool* dir) {
  const int d = slot >> 1, s = slot & 1;
  const long long n2 = (long long)g.n * g.n;
  if (d == 0) {
    const int f = ex + s;
    *dir = (f == 0 || f == g.mx);
    return sem_dbg_entity(g.off[0] + (f + (long long)(g.mx + 1) * (ey + (long long)g.my * ez)) * n2, n2, g, dir);
  }
  if (d == 1) {
    const int f = ey + s;
    *dir = (f == 0 || f == g.my);
    return sem_dbg_entity(g.off[1] + (ex + (long long)g.mx * (f + (long long)(g.my + 1) * ez)) * n2, n2, g, dir);
  }
  const int f = ez + s;
  *dir = (f == 0 || f == g.mz);
  return sem_dbg_entity(g.off[2] + (ex + (long long)g.mx * (ey + (long long)g.my * f)) * n2, n2, g, dir);
}

// Edge slot 0..11: group = slot >> 2 (0 x-edges Ex[sb][sc], 1 y-edges Ey[sa][sc],
// 2 z-edges Ez[sa][sb]); the two side bits are slot & 1 and (slot >> 1) & 1.
static __device__ __forceinline__ long long edge_base(const SemGeom& g, int ex, int ey, int ez, int slot, bool* dir) {
  const int grp = slot >> 2, s1 = slot & 1, s2 = (slot >> 1) & 1;
  if (grp == 0) {
    const int vy = ey + s1, vz = ez + s2;
    *dir = (vy == 0 || vy == g.my || vz == 0 || vz == g.mz);
    return sem_dbg_entity(g.off[3] + (ex + (long long)g.mx * (vy + (long long)(g.my + 1) * vz)) * g.n, g.n, g, dir);
  }
  if (grp == 1) {
    const int vx = ex + s1, vz = ez + s2;
    *dir = (vx == 0 || vx == g.mx || vz == 0 || vz == g.mz);
    return sem_dbg_entity(g.off[4] + (vx + (long long)(g.mx + 1) * (ey + (long long)g.my * vz)) * g.n, g.n, g, dir);
  }
  const int vx = ex + s1, vy = ey + s2;
  *dir = (vx == 0 || vx == g.mx || vy == 0 || vy == g.my);
  return sem_dbg_entity(g.off[5] + (vx + (long long)(g.mx + 1) * (vy + (long long)(g.my + 1) * ez)) * g.n, g.n, g, dir);
}

// Vertex slot 0..7 = sa + 2 sb + 4 sc.
static __device__ __forceinline__ long long vert_index(const SemGeom& g, int ex, int ey, int ez, int slot, bool* dir) {
  const int vx = ex + (slot & 1), vy = ey + ((slot >> 1) & 1), vz = ez + (slot >> 2);
  *dir = (vx == 0 || vx == g.mx || vy == 0 || vy == g.my || vz == 0 || vz == g.mz);
  return sem_dbg_entity(g.off[6] + vx + (long long)(g.mx + 1) * (vy + (long long)(g.my + 1) * vz), 1, g, dir);
}

// Entity offsets are affine in the element coordinates: offset of entity
// slot r = base + ex sx + ey sy + ez sz, and the entity is on the Dirichlet
// boundary iff one of the element's boundary flags in `mask` is set (bit 2a:
// coordinate a is 0, bit 2a + 1: coordinate a is m_a - 1).  Slots as in
// face_base / edge_base / vert_index (sem_device.cuh).
struct EntityAffine {
  int base, sx, sy, sz, mask;
};

static __device__ void entity_affine(const SemGeom& g, int r, EntityAffine* out) {
  const int n = g.n, n2 = n * n, mx = g.mx, my = g.my;
  EntityAffine a;
  if (r < 6) {
    const int d = r >> 1, s = r & 1;
    a.sx = n2;
    if (d == 0) { a.base = (int)g.off[0] + s * n2; a.sy = (mx + 1) * n2; a.sz = (mx + 1) * my * n2; }
    else if (d == 1) { a.base = (int)g.off[1] + s * mx * n2; a.sy = mx * n2; a.sz = mx * (my + 1) * n2; }
    else { a.base = (int)g.off[2] + s * mx * my * n2; a.sy = mx * n2; a.sz = mx * my * n2; }
    a.mask = 1 << (2 * d + s);
  } else if (r < 18) {
    const int q = r - 6, grp = q >> 2, s1 = q & 1, s2 = (q >> 1) & 1;
    a.sx = n;
    if (grp == 0) {        // x-edge (sb, sc) = (s1, s2): y and z shifted
      a.base = (int)g.off[3] + (mx * s1 + mx * (my + 1) * s2) * n; a.sy = mx * n; a.sz = mx * (my + 1) * n;
      a.mask = (1 << (2 + s1)) | (1 << (4 + s2));
    } else if (grp == 1) { // y-edge (sa, sc): x and z shifted
      a.base = (int)g.off[4] + (s1 + (mx + 1) * my * s2) * n; a.sy = (mx + 1) * n; a.sz = (mx + 1) * my * n;
      a.mask = (1 << s1) | (1 << (4 + s2));
    } else {               // z-edge (sa, sb): x and y shifted
      a.base = (int)g.off[5] + (s1 + (mx + 1) * s2) * n; a.sy = (mx + 1) * n; a.sz = (mx + 1) * (my + 1) * n;
      a.mask = (1 << s1) | (1 << (2 + s2));
    }
  } else {
    const int q = r - 18, sa = q & 1, sb = (q >> 1) & 1, sc = q >> 2;
    a.base = (int)g.off[6] + sa + (mx + 1) * sb + (mx + 1) * (my + 1) * sc;
    a.sx = 1;
    a.sy = mx + 1;
    a.sz = (mx + 1) * (my + 1);
    a.mask = (1 << sa) | (1 << (2 + sb)) | (1 << (4 + sc));
  }
  *out = a;
}

// Offset of entity slot r of an element with boundary flags `bits` from the
// affine form (-1: Dirichlet entity); debug builds check it as sem_dbg_entity.
static __device__ __forceinline__ int entity_offset(const EntityAffine& a, int r, int bits, int ex, int ey, int ez,
                                                    const SemGeom& g) {
#ifdef SEM_DEBUG
  bool dir = (bits & a.mask) != 0;
  const int off = a.base + ex * a.sx + ey * a.sy + ez * a.sz;
  sem_dbg_entity(off, r < 6 ? (long long)g.n * g.n : (r < 18 ? g.n : 1), g, &dir);
  return dir ? -1 : off;
#else
  (void)r; (void)g;
  return (bits & a.mask) ? -1 : a.base + ex * a.sx + ey * a.sy + ez * a.sz;
#endif
}

template <typename T>
static __device__ __forceinline__ int elem_class(const SemGeom& g, const SemClassTables<T>& t, int ex, int ey, int ez) {
#ifdef SEM_DEBUG
  const int c = t.cls_x[ex] + g.ux * (t.cls_y[ey] + g.uy * t.cls_z[ez]);
  return sem_dbg_ok(c, 1, (long long)g.ux * g.uy * g.uz) ? c : 0;
#else
  return t.cls_x[ex] + g.ux * (t.cls_y[ey] + g.uy * t.cls_z[ez]);
#endif
}

// Global node (gx, gy, gz) of packed skeleton entry idx.
static __device__ __forceinline__ void skel_node(const SemGeom& g, long long idx, long long* gx, long long* gy,
                                          long long* gz) {
  const int p = g.p, n = g.n;
  const long long n2 = (long long)n * n;
  int b = 0;
  while (b < 6 && idx >= g.off[b + 1]) ++b;
  const long long loc = idx - g.off[b];
  if (b < 3) {
    const long long ent = loc / n2, r = loc - ent * n2;
    const int fast = (int)(r % n) + 1, slow = (int)(r / n) + 1;
    if (b == 0) {
      const long long f = ent % (g.mx + 1), t = ent / (g.mx + 1);
      *gx = f * p; *gy = (t % g.my) * p + fast; *gz = (t / g.my) * p + slow;
    } else if (b == 1) {
      const long long ex = ent % g.mx, t = ent / g.mx;
      *gx = ex * p + fast; *gy = (t % (g.my + 1)) * p; *gz = (t / (g.my + 1)) * p + slow;
    } else {
      const long long ex = ent % g.mx, t = ent / g.mx;
      *gx = ex * p + fast; *gy = (t % g.my) * p + slow; *gz = (t / g.my) * p;
    }
  } else if (b < 6) {
    const long long ent = loc / n;
    const int l = (int)(loc - ent * n) + 1;
    if (b == 3) {
      const long long ex = ent % g.mx, t = ent / g.mx;
      *gx = ex * p + l; *gy = (t % (g.my + 1)) * p; *gz = (t / (g.my + 1)) * p;
    } else if (b == 4) {
      const long long vx = ent % (g.mx + 1), t = ent / (g.mx + 1);
      *gx = vx * p; *gy = (t % g.my) * p + l; *gz = (t / g.my) * p;
    } else {
      const long long vx = ent % (g.mx + 1), t = ent / (g.mx + 1);
      *gx = vx * p; *gy = (t % (g.my + 1)) * p; *gz = (t / (g.my + 1)) * p + l;
    }
  } else {
    const long long vx = loc % (g.mx + 1), t = loc / (g.mx + 1);
    *gx = vx * p; *gy = (t % (g.my + 1)) * p; *gz = (t / (g.my + 1)) * p;
  }
}

static __device__ __forceinline__ bool node_on_boundary(const SemGeom& g, long long gx, long long gy, long long gz) {
  return gx == 0 || gx == g.Nx - 1 || gy == 0 || gy == g.Ny - 1 || gz == 0 || gz == g.Nz - 1;
}

// ---------------------------------------------------------------------------
// Deterministic block reduction + last-block finalisation
// ---------------------------------------------------------------------------
template <int NV>
static __device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /* [NV][32] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[k * 32 + wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = lane < nw ? sh[k * 32 + lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[k] = x;   // valid in thread 0
    }
  }
  __syncthreads();
}

// Writes this block's NV sums to partials[k * G + block]; the last block to
// arrive sums all partials in a fixed order and returns true with the totals
// in tot (valid in thread 0).
template <int NV>
static __device__ bool reduce_grid(double (&v)[NV], double* partials, unsigned int* counter, double (&tot)[NV]) {
  __shared__ double sh[NV * 32];
  __shared__ bool last;
  block_sum<NV>(v, sh);
  const unsigned G = gridDim.x;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[k * G + blockIdx.x] = v[k];
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    last = (t == G - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    s[k] = 0.0;
    for (unsigned i = threadIdx.x; i < G; i += blockDim.x) s[k] += __ldcg(partials + k * G + i);
  }
  block_sum<NV>(s, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = s[k];
    *counter = 0u;
  }
  return true;
}

// 1/x to within 1 ulp (FP32, flush-to-zero), one MUFU instruction.
static __device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// cp.async of 4 bytes global -> shared; zero-fills the destination when
// !valid (src-size 0: nothing is read).
static __device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
// cp.async of 16 bytes (both addresses 16-byte aligned).
static __device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
static __device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
static __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory"); }

}  // namespace semdev

// Host reader of one translation unit's bounds record (debug builds): adds its
// count to *count, keeps its first offending value in *first if none was kept
// yet, and clears the record.  Expands to nothing in release builds.
#ifdef SEM_DEBUG
#define SEM_DEBUG_TU(tag)                                                                  \
  cudaError_t sem_debug_take_##tag(unsigned long long* count, long long* first) {          \
    unsigned long long c = 0;                                                              \
    long long f = 0;                                                                       \
    cudaError_t e = cudaMemcpyFromSymbol(&c, semdev::sem_dbg_count, sizeof c);             \
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&f, semdev::sem_dbg_first, sizeof f);   \
    if (e != cudaSuccess) return e;                                                        \
    if (c != 0 && *count == 0) *first = f;                                                 \
    *count += c;                                                                           \
    const unsigned long long z = 0;                                                        \
    return cudaMemcpyToSymbol(semdev::sem_dbg_count, &z, sizeof z);                        \
  }
#else
#define SEM_DEBUG_TU(tag)
#endif
