// The transformed condensed operator, fused over gather, primary part,
// condensed part and scatter (Sec. 6 of the paper).
//
//   v~ = sum_e Rhat_e (H~_BB - H~_BI D^-1 H~_IB) Rhat_e^T u~
//
// * Condensed part (Table 2): the six faces are expanded into the interior
//   eigenspace with d K~_{I0}, d K~_{Ip} (one rank-1 term per face and line),
//   scaled by D^-1 (Eq. hii_diagonal) and contracted back with d K~_{0I},
//   d K~_{pI}: 6 n^3 + n^3 + 6 n^3 multiply-adds (Table 3's 13 n^3).
// * Primary part H~_BB: the restriction of
//   H~ = d0 M~(x)M~(x)M~ + d1 M~(x)M~(x)K~ + d2 M~(x)K~(x)M~ + d3 K~(x)M~(x)M~
//   to the skeleton, M~ = diag(w0, I, w0), K~ = S K S^T.  Face self-blocks are
//   diagonal (Eq. east_east_primary_part_transformed); only 1D lines lying in
//   a face or along an edge couple different entities.
// * Gather R^T and scatter-add R: faces have 2 contributions, edges 4,
//   vertices 8 (reductions in L2 with red.global.add).
//
// GB300 mapping: one CTA works on a tile of `epb` elements held entirely in
// shared memory (faces, edges, vertices, outputs, a k-slab of the n^3 cube).
// Entity offsets are computed once per element, coefficient vectors come from
// per-width-class tables (reloaded only when the class changes: elements are
// visited with the most-graded axis slowest, and each CTA takes a contiguous
// range of tiles), and every item loop is uniform in its branch so warps stay
// converged.  The degree is a template parameter for the common p.
#include <cuda_runtime.h>

#include "sem_device.cuh"
#include "sem_kernels.cuh"

using namespace semdev;

namespace {

constexpr int kThreads = 256;
constexpr int kHdrInts = 28;   // per element: class, loaded class, 6 + 12 + 8 entity offsets

// Shared-memory layout of one element (units of T).
struct ElemSm {
  int F, Acc, E, Eo, Vt, Vo, C, Bt, cube, size;
};

__host__ __device__ inline ElemSm elem_sm(int n, int ks) {
  const int n2 = n * n;
  ElemSm L;
  L.F = 0;
  L.Acc = 6 * n2;
  L.E = 12 * n2;
  L.Eo = L.E + 12 * n;
  L.Vt = L.Eo + 12 * n;
  L.Vo = L.Vt + 8;
  L.C = L.Vo + 8;
  L.Bt = L.C + 18 * n + 24;     // b/t contractions (summed over all k-slabs)
  L.cube = L.Bt + 2 * n2;
  L.size = (L.cube + ks * n2 + 3) & ~3;
  return L;
}

__host__ __device__ inline size_t hdr_bytes(int epb) { return ((size_t)epb * kHdrInts * 4 + 31) & ~size_t(31); }

// ---------------------------------------------------------------------------
// Per-class coefficient blocks
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_class_coeffs(SemGeom g, SemBasis b, const double* __restrict__ dcoef,
                               const double* __restrict__ dinv, T* __restrict__ coef) {
  const int n = g.n, n2 = n * n;
  const CoefOffsets o = coef_offsets(n);
  const long long ncls = (long long)g.ux * g.uy * g.uz;
  const double w0 = b.w0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncls * o.stride;
       t += (long long)gridDim.x * blockDim.x) {
    const long long c = t / o.stride;
    const int r = (int)(t - c * o.stride);
    const double* d = dcoef + c * 4;
    double v = 0.0;
    if (r < 18 * n) {                       // skd, skw, skww
      const int which = r / (6 * n), q = r - which * 6 * n, ds = q / n, i = q - ds * n;
      const double sc = which == 0 ? 1.0 : (which == 1 ? w0 : w0 * w0);
      v = d[(ds >> 1) + 1] * sc * b.k[ds & 1][i];
    } else if (r < 18 * n + 18) {           // cO, eO, vO
      const int q = r - 18 * n, which = q / 6, ds = q - which * 6, s = ds & 1;
      const double sc = which == 0 ? 1.0 : (which == 1 ? w0 : w0 * w0);
      v = d[(ds >> 1) + 1] * sc * b.K[s][1 - s];
    } else if (r < o.fdiag) {
      v = 0.0;
    } else if (r < o.ediag) {               // face diagonals
      const int q = r - o.fdiag, slot = q / n2, idx = q - slot * n2, dd = slot >> 1, s = slot & 1;
      const int slow = idx / n, fast = idx - slow * n;
      const double Kss = b.K[s][s];
      if (dd == 0) v = d[0] * w0 + d[1] * Kss + w0 * (d[2] * b.lam[fast] + d[3] * b.lam[slow]);
      else if (dd == 1) v = d[0] * w0 + d[2] * Kss + w0 * (d[1] * b.lam[fast] + d[3] * b.lam[slow]);
      else v = d[0] * w0 + d[3] * Kss + w0 * (d[1] * b.lam[fast] + d[2] * b.lam[slow]);
    } else if (r < o.vdiag) {               // edge diagonals
      const int q = r - o.ediag, slot = q / n, l = q - slot * n;
      const int grp = slot >> 2, s1 = slot & 1, s2 = (slot >> 1) & 1;
      const int t1 = grp == 0 ? 1 : 0, t2 = grp == 2 ? 1 : 2;
      v = d[0] * w0 * w0 + d[grp + 1] * w0 * w0 * b.lam[l] + d[t1 + 1] * w0 * b.K[s1][s1] +
          d[t2 + 1] * w0 * b.K[s2][s2];
    } else if (r < o.vdiag + 8) {           // vertex diagonals
      const int slot = r - o.vdiag, sa = slot & 1, sb = (slot >> 1) & 1, sc = slot >> 2;
      v = d[0] * w0 * w0 * w0 + w0 * w0 * (d[1] * b.K[sa][sa] + d[2] * b.K[sb][sb] + d[3] * b.K[sc][sc]);
    } else if (r >= o.ndinv && r < o.ndinv + n2 * n) {
      v = -dinv[c * n2 * n + (r - o.ndinv)];
    }
    coef[t] = (T)v;
  }
}

// ---------------------------------------------------------------------------
// The operator kernel
// ---------------------------------------------------------------------------
template <typename T, int NC>
__global__ void __launch_bounds__(kThreads)
k_tpt_apply(SemGeom g, SemClassTables<T> tab, const T* __restrict__ u, T* __restrict__ v, int epb, int ks,
            double* __restrict__ partials, PcgState* st, T* __restrict__ ev) {
  extern __shared__ __align__(32) unsigned char smem_raw[];
  if (st != nullptr && st->done) return;
  const int n = NC > 0 ? NC : g.n;
  const int n2 = n * n;
  const ElemSm L = elem_sm(n, ks);
  const CoefOffsets co = coef_offsets(n);
  int* hdr = reinterpret_cast<int*>(smem_raw);                 // [epb][kHdrInts]
  T* elems = reinterpret_cast<T*>(smem_raw + hdr_bytes(epb));
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int t = tid; t < epb; t += nt) hdr[t * kHdrInts + 1] = -1;   // no class loaded yet
  const long long ntiles = (g.nelem + epb - 1) / epb;
  const long long t_begin = ntiles * blockIdx.x / gridDim.x;
  const long long t_end = ntiles * (blockIdx.x + 1) / gridDim.x;
  T dot = T(0);

  for (long long tile = t_begin; tile < t_end; ++tile) {
    const long long e0 = tile * epb;
    __syncthreads();
    // ---- element headers: class and entity offsets (-1 on the Dirichlet boundary)
    for (int t = tid; t < epb * 26; t += nt) {
      const int el = t / 26, r = t - el * 26;
      const long long e = e0 + el;
      int* h = hdr + el * kHdrInts;
      if (e >= g.nelem) {
        if (r == 0) h[0] = -2;
        h[2 + r] = -1;
        continue;
      }
      int ex, ey, ez;
      elem_visit(g, e, &ex, &ey, &ez);
      bool dir;
      long long off;
      if (r < 6) off = face_base(g, ex, ey, ez, r, &dir);
      else if (r < 18) off = edge_base(g, ex, ey, ez, r - 6, &dir);
      else off = vert_index(g, ex, ey, ez, r - 18, &dir);
      h[2 + r] = dir ? -1 : (int)off;
      if (r == 0) h[0] = elem_class(g, tab, ex, ey, ez);
    }
    __syncthreads();
    // ---- gather R^T and the class coefficient vectors
    for (int t = tid; t < epb * 6 * n2; t += nt) {
      const int el = t / (6 * n2), r = t - el * 6 * n2, slot = r / n2, idx = r - slot * n2;
      const int off = hdr[el * kHdrInts + 2 + slot];
      elems[el * L.size + L.F + r] = off >= 0 ? u[off + idx] : T(0);
    }
    for (int t = tid; t < epb * 12 * n; t += nt) {
      const int el = t / (12 * n), r = t - el * 12 * n, slot = r / n, l = r - slot * n;
      const int off = hdr[el * kHdrInts + 8 + slot];
      elems[el * L.size + L.E + r] = off >= 0 ? u[off + l] : T(0);
    }
    for (int t = tid; t < epb * 8; t += nt) {
      const int el = t >> 3, r = t & 7;
      const int off = hdr[el * kHdrInts + 20 + r];
      elems[el * L.size + L.Vt + r] = off >= 0 ? u[off] : T(0);
    }
    for (int t = tid; t < epb * (18 * n + 18); t += nt) {
      const int el = t / (18 * n + 18), r = t - el * (18 * n + 18);
      const int* h = hdr + el * kHdrInts;
      if (h[0] >= 0 && h[0] != h[1]) elems[el * L.size + L.C + r] = tab.coef[(long long)h[0] * co.stride + r];
    }
    __syncthreads();
    for (int t = tid; t < epb; t += nt) hdr[t * kHdrInts + 1] = hdr[t * kHdrInts];

    // ---- primary part on faces -> Acc (one loop per direction: uniform branches)
#pragma unroll 1
    for (int dd = 0; dd < 3; ++dd) {
      for (int t = tid; t < epb * 2 * n2; t += nt) {
        const int el = t / (2 * n2), r = t - el * 2 * n2, s = r / n2, idx = r - s * n2;
        const int slow = idx / n, fast = idx - slow * n;
        T* E = elems + el * L.size;
        const int cls = hdr[el * kHdrInts];
        if (cls < 0) continue;
        const T* F = E + L.F;
        const T* Ed = E + L.E;
        const T* skw = E + L.C + 6 * n;
        const T* cO = E + L.C + 18 * n;
        const int slot = 2 * dd + s;
        const T diag = __ldg(tab.coef + (long long)cls * co.stride + co.fdiag + slot * n2 + idx);
        T out = diag * F[slot * n2 + idx];
        out = fma(cO[slot], F[(slot ^ 1) * n2 + idx], out);
        if (dd == 0) {          // x-face, (j, k) = (fast, slow)
          const int j = fast, k = slow;
          out = fma(skw[2 * n + j], Ed[(8 + s) * n + k], out);        // Ez[s][0]
          out = fma(skw[3 * n + j], Ed[(10 + s) * n + k], out);       // Ez[s][1]
          out = fma(skw[4 * n + k], Ed[(4 + s) * n + j], out);        // Ey[s][0]
          out = fma(skw[5 * n + k], Ed[(6 + s) * n + j], out);        // Ey[s][1]
        } else if (dd == 1) {   // y-face, (i, k)
          const int i = fast, k = slow;
          out = fma(skw[0 * n + i], Ed[(8 + 2 * s) * n + k], out);    // Ez[0][s]
          out = fma(skw[1 * n + i], Ed[(9 + 2 * s) * n + k], out);    // Ez[1][s]
          out = fma(skw[4 * n + k], Ed[(0 + s) * n + i], out);        // Ex[s][0]
          out = fma(skw[5 * n + k], Ed[(2 + s) * n + i], out);        // Ex[s][1]
        } else {                // z-face, (i, j)
          const int i = fast, j = slow;
          out = fma(skw[0 * n + i], Ed[(4 + 2 * s) * n + j], out);    // Ey[0][s]
          out = fma(skw[1 * n + i], Ed[(5 + 2 * s) * n + j], out);    // Ey[1][s]
          out = fma(skw[2 * n + j], Ed[(0 + 2 * s) * n + i], out);    // Ex[0][s]
          out = fma(skw[3 * n + j], Ed[(1 + 2 * s) * n + i], out);    // Ex[1][s]
        }
        E[L.Acc + slot * n2 + idx] = out;
      }
    }
    // ---- primary part on edges -> Eo
#pragma unroll 1
    for (int grp = 0; grp < 3; ++grp) {
      for (int t = tid; t < epb * 4 * n; t += nt) {
        const int el = t / (4 * n), r = t - el * 4 * n, q = r / n, l = r - q * n;
        const int s1 = q & 1, s2 = q >> 1, slot = 4 * grp + q;
        T* E = elems + el * L.size;
        const int cls = hdr[el * kHdrInts];
        if (cls < 0) continue;
        const T* F = E + L.F;
        const T* Ed = E + L.E;
        const T* Vt = E + L.Vt;
        const T* skw = E + L.C + 6 * n;
        const T* skww = E + L.C + 12 * n;
        const T* eO = E + L.C + 18 * n + 6;
        const T diag = __ldg(tab.coef + (long long)cls * co.stride + co.ediag + slot * n + l);
        T out = diag * Ed[slot * n + l];
        if (grp == 0) {         // x-edge Ex[sb][sc], index i
          const int sb = s1, sc = s2, i = l;
          out = fma(skww[i], Vt[2 * sb + 4 * sc], out);
          out = fma(skww[n + i], Vt[1 + 2 * sb + 4 * sc], out);
          const T* kb = skw + (2 + sb) * n;
          const T* kc = skw + (4 + sc) * n;
          const T* Fz = F + (4 + sc) * n2 + i;
          const T* Fy = F + (2 + sb) * n2 + i;
#pragma unroll 4
          for (int m = 0; m < n; ++m) out = fma(kb[m], Fz[m * n], out);
#pragma unroll 4
          for (int m = 0; m < n; ++m) out = fma(kc[m], Fy[m * n], out);
          out = fma(eO[2 + sb], Ed[((1 - sb) + 2 * sc) * n + i], out);
          out = fma(eO[4 + sc], Ed[(sb + 2 * (1 - sc)) * n + i], out);
        } else if (grp == 1) {  // y-edge Ey[sa][sc], index j
          const int sa = s1, sc = s2, j = l;
          out = fma(skww[2 * n + j], Vt[sa + 4 * sc], out);
          out = fma(skww[3 * n + j], Vt[sa + 2 + 4 * sc], out);
          const T* ka = skw + sa * n;
          const T* kc = skw + (4 + sc) * n;
          const T* Fz = F + (4 + sc) * n2 + j * n;
          const T* Fx = F + sa * n2 + j;
#pragma unroll 4
          for (int m = 0; m < n; ++m) out = fma(ka[m], Fz[m], out);
#pragma unroll 4
          for (int m = 0; m < n; ++m) out = fma(kc[m], Fx[m * n], out);
          out = fma(eO[sa], Ed[(4 + (1 - sa) + 2 * sc) * n + j], out);
          out = fma(eO[4 + sc], Ed[(4 + sa + 2 * (1 - sc)) * n + j], out);
        } else {                // z-edge Ez[sa][sb], index k
          const int sa = s1, sb = s2, k = l;
          out = fma(skww[4 * n + k], Vt[sa + 2 * sb], out);
          out = fma(skww[5 * n + k], Vt[sa + 2 * sb + 4], out);
          const T* ka = skw + sa * n;
          const T* kb = skw + (2 + sb) * n;
          const T* Fy = F + (2 + sb) * n2 + k * n;
          const T* Fx = F + sa * n2 + k * n;
#pragma unroll 4
          for (int m = 0; m < n; ++m) out = fma(ka[m], Fy[m], out);
#pragma unroll 4
          for (int m = 0; m < n; ++m) out = fma(kb[m], Fx[m], out);
          out = fma(eO[sa], Ed[(8 + (1 - sa) + 2 * sb) * n + k], out);
          out = fma(eO[2 + sb], Ed[(8 + sa + 2 * (1 - sb)) * n + k], out);
        }
        E[L.Eo + slot * n + l] = out;
      }
    }
    // ---- primary part at vertices -> Vo
    for (int t = tid; t < epb * 8; t += nt) {
      const int el = t >> 3, slot = t & 7;
      const int sa = slot & 1, sb = (slot >> 1) & 1, sc = slot >> 2;
      T* E = elems + el * L.size;
      const int cls = hdr[el * kHdrInts];
      if (cls < 0) continue;
      const T* Ed = E + L.E;
      const T* Vt = E + L.Vt;
      const T* skww = E + L.C + 12 * n;
      const T* vO = E + L.C + 18 * n + 12;
      const T diag = __ldg(tab.coef + (long long)cls * co.stride + co.vdiag + slot);
      T out = diag * Vt[slot];
      const T* ka = skww + sa * n;
      const T* kb = skww + (2 + sb) * n;
      const T* kc = skww + (4 + sc) * n;
      const T* exl = Ed + (sb + 2 * sc) * n;
      const T* eyl = Ed + (4 + sa + 2 * sc) * n;
      const T* ezl = Ed + (8 + sa + 2 * sb) * n;
      for (int m = 0; m < n; ++m) out = fma(ka[m], exl[m], out);
      for (int m = 0; m < n; ++m) out = fma(kb[m], eyl[m], out);
      for (int m = 0; m < n; ++m) out = fma(kc[m], ezl[m], out);
      out = fma(vO[sa], Vt[slot ^ 1], out);
      out = fma(vO[2 + sb], Vt[slot ^ 2], out);
      out = fma(vO[4 + sc], Vt[slot ^ 4], out);
      E[L.Vo + slot] = out;
    }

    // ---- condensed part, one k-slab of the eigenspace cube at a time.
    // Expansion (Table 2) and -D^-1: one thread per (j, i) column of the cube,
    // face values and scaled vectors of the column held in registers; the b/t
    // contraction (sum over k) is done in the same registers.
    for (int k0 = 0; k0 < n; k0 += ks) {
      const int kn = min(ks, n - k0);
      for (int t = tid; t < epb * n2; t += nt) {
        const int el = t / n2, ji = t - el * n2, j = ji / n, i = ji - j * n;
        T* E = elems + el * L.size;
        const int cls = hdr[el * kHdrInts];
        const T* F = E + L.F;
        const T* skd = E + L.C;
        const T ai = skd[i], bi = skd[n + i], cj = skd[2 * n + j], dj = skd[3 * n + j];
        const T fb = F[4 * n2 + ji], ft = F[5 * n2 + ji];
        const T* nd = tab.coef + (cls >= 0 ? (long long)cls * co.stride : 0LL) + co.ndinv + ji;
        T sb = k0 == 0 ? T(0) : E[L.Bt + ji];
        T st_ = k0 == 0 ? T(0) : E[L.Bt + n2 + ji];
        T* cube = E + L.cube + ji;
#pragma unroll 4
        for (int kk = 0; kk < kn; ++kk) {
          const int k = k0 + kk;
          const T ek = skd[4 * n + k], gk = skd[5 * n + k];
          T x = ai * F[k * n + j];
          x = fma(bi, F[n2 + k * n + j], x);
          x = fma(cj, F[2 * n2 + k * n + i], x);
          x = fma(dj, F[3 * n2 + k * n + i], x);
          x = fma(ek, fb, x);
          x = fma(gk, ft, x);
          const T vv = (cls >= 0 ? __ldg(nd + k * n2) : T(0)) * x;
          cube[kk * n2] = vv;
          sb = fma(ek, vv, sb);
          st_ = fma(gk, vv, st_);
        }
        E[L.Bt + ji] = sb;
        E[L.Bt + n2 + ji] = st_;
      }
      __syncthreads();
      // w / e: rows over i, both faces from one pass over the row
      for (int t = tid; t < epb * kn * n; t += nt) {
        const int el = t / (kn * n), q = t - el * kn * n, kk = q / n, j = q - kk * n;
        T* E = elems + el * L.size;
        const T* ka = E + L.C;
        const T* kb = E + L.C + n;
        const T* row = E + L.cube + kk * n2 + j * n;
        const int o = (k0 + kk) * n + j;
        T s0 = E[L.Acc + o], s1 = E[L.Acc + n2 + o];
#pragma unroll 8
        for (int i = 0; i < n; ++i) {
          const T c = row[i];
          s0 = fma(ka[i], c, s0);
          s1 = fma(kb[i], c, s1);
        }
        E[L.Acc + o] = s0;
        E[L.Acc + n2 + o] = s1;
      }
      // s / n: columns over j
      for (int t = tid; t < epb * kn * n; t += nt) {
        const int el = t / (kn * n), q = t - el * kn * n, kk = q / n, i = q - kk * n;
        T* E = elems + el * L.size;
        const T* ka = E + L.C + 2 * n;
        const T* kb = E + L.C + 3 * n;
        const T* col = E + L.cube + kk * n2 + i;
        const int o = (k0 + kk) * n + i;
        T s0 = E[L.Acc + 2 * n2 + o], s1 = E[L.Acc + 3 * n2 + o];
#pragma unroll 8
        for (int j = 0; j < n; ++j) {
          const T c = col[j * n];
          s0 = fma(ka[j], c, s0);
          s1 = fma(kb[j], c, s1);
        }
        E[L.Acc + 2 * n2 + o] = s0;
        E[L.Acc + 3 * n2 + o] = s1;
      }
      __syncthreads();
    }

    // ---- scatter R and the element share of x^T (A x)
    for (int t = tid; t < epb * 6 * n2; t += nt) {
      const int el = t / (6 * n2), r = t - el * 6 * n2, slot = r / n2, idx = r - slot * n2;
      const int off = hdr[el * kHdrInts + 2 + slot];
      if (off < 0) continue;
      const T* E = elems + el * L.size;
      const T o = slot >= 4 ? E[L.Acc + r] + E[L.Bt + r - 4 * n2] : E[L.Acc + r];
      atomicAdd(v + off + idx, o);
      dot = fma(E[L.F + r], o, dot);
    }
    for (int t = tid; t < epb * 12 * n; t += nt) {
      const int el = t / (12 * n), r = t - el * 12 * n, slot = r / n, l = r - slot * n;
      const int off = hdr[el * kHdrInts + 8 + slot];
      if (off < 0) continue;
      const T* E = elems + el * L.size;
      const T o = E[L.Eo + r];
      // fixed-order mode: the element's share goes to its slot, summed by k_ev_sum
      if (ev != nullptr) ev[(e0 + el) * (12LL * n + 8) + r] = o;
      else atomicAdd(v + off + l, o);
      dot = fma(E[L.E + r], o, dot);
    }
    for (int t = tid; t < epb * 8; t += nt) {
      const int el = t >> 3, r = t & 7;
      const int off = hdr[el * kHdrInts + 20 + r];
      if (off < 0) continue;
      const T* E = elems + el * L.size;
      const T o = E[L.Vo + r];
      if (ev != nullptr) ev[(e0 + el) * (12LL * n + 8) + 12 * n + r] = o;
      else atomicAdd(v + off, o);
      dot = fma(E[L.Vt + r], o, dot);
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

int num_sms_cached() { return sem_num_sms(); }

// ---------------------------------------------------------------------------
// Warp-per-element variant for small degrees (n <= 7)
// ---------------------------------------------------------------------------
// One warp owns one element at a time: its whole working set sits in the
// warp's slice of shared memory and phases are separated by __syncwarp only,
// so warps of a CTA progress independently.  Trip counts are compile-time.
template <int N>
struct WarpSm {
  static constexpr int N2 = N * N, N3 = N2 * N, RS = (N + 3) & ~3;   // cube rows padded to 4
  static constexpr int F = 0, E = 6 * N2, Vt = E + 12 * N, C = Vt + 8, P2 = C + 18 * N + 24,
                       cube = (P2 + 6 * N + 3) & ~3, size = (cube + N2 * RS + 3) & ~3;
};
constexpr int kWarpHdr = 32;   // ints per warp: 26 entity offsets, class, loaded class

template <typename T>
struct Two {
  T x, y;
};

// The face primary part is evaluated where its inputs already sit in
// registers: z-faces in the cube-column loop, x- and y-faces in the
// contraction loop; every face output goes to the skeleton straight from
// registers.  skw = w0 * skd is used for the in-face line couplings.
template <typename T, int N>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2)
k_tpt_apply_warp(SemGeom g, SemClassTables<T> tab, const T* __restrict__ u, T* __restrict__ v,
                 double* __restrict__ partials, PcgState* st, T w0) {
  using S = WarpSm<N>;
  constexpr int N2 = S::N2, RS = S::RS;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  if (st != nullptr && st->done) return;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  int* H = reinterpret_cast<int*>(smem_raw) + wib * kWarpHdr;
  T* W = reinterpret_cast<T*>(smem_raw + ((size_t)wpb * kWarpHdr * 4 + 31) / 32 * 32) + (size_t)wib * S::size;
  const CoefOffsets co = coef_offsets(N);
  const long long nwarps = (long long)gridDim.x * wpb, gw = (long long)blockIdx.x * wpb + wib;
  const long long e_begin = g.nelem * gw / nwarps, e_end = g.nelem * (gw + 1) / nwarps;
  if (lane == 0) H[27] = -1;
  T dot = T(0);
  const int mx = g.mx, my = g.my, mz = g.mz;
  const Two<T>* P2 = reinterpret_cast<const Two<T>*>(W + S::P2);   // [dir][t]: (skd[2dir N + t], skd[(2dir+1) N + t])

  for (long long e = e_begin; e < e_end; ++e) {
    int ex, ey, ez;
    {
      const int ei = (int)e;
      if (g.slow == 0) { ex = ei / (my * mz); const int r = ei - ex * (my * mz); ey = r % my; ez = r / my; }
      else if (g.slow == 1) { ey = ei / (mx * mz); const int r = ei - ey * (mx * mz); ex = r % mx; ez = r / mx; }
      else { ex = ei % mx; const int r = ei / mx; ey = r % my; ez = r / my; }
    }
    __syncwarp();
    if (lane < 26) {
      bool dir;
      long long off;
      if (lane < 6) off = face_base(g, ex, ey, ez, lane, &dir);
      else if (lane < 18) off = edge_base(g, ex, ey, ez, lane - 6, &dir);
      else off = vert_index(g, ex, ey, ez, lane - 18, &dir);
      H[lane] = dir ? -1 : (int)off;
    } else if (lane == 26) {
      H[26] = elem_class(g, tab, ex, ey, ez);
    }
    __syncwarp();
    const int cls = H[26];
    const T* cb = tab.coef + (long long)cls * co.stride;
    // gather R^T
#pragma unroll
    for (int r = lane; r < 6 * N2; r += 32) {
      const int slot = r / N2, off = H[slot];
      W[S::F + r] = off >= 0 ? u[off + r - slot * N2] : T(0);
    }
#pragma unroll
    for (int r = lane; r < 12 * N; r += 32) {
      const int slot = r / N, off = H[6 + slot];
      W[S::E + r] = off >= 0 ? u[off + r - slot * N] : T(0);
    }
    if (lane < 8) {
      const int off = H[18 + lane];
      W[S::Vt + lane] = off >= 0 ? u[off] : T(0);
    }
    if (cls != H[27]) {
      for (int r = lane; r < 18 * N + 18; r += 32) W[S::C + r] = cb[r];
      for (int r = lane; r < 6 * N; r += 32) {
        const int dir = r / (2 * N), rem = r - dir * 2 * N, t = rem >> 1, side = rem & 1;
        W[S::P2 + r] = cb[(2 * dir + side) * N + t];
      }
    }
    __syncwarp();
    if (lane == 0) H[27] = cls;
    const T* F = W + S::F;
    const T* Ed = W + S::E;
    const T* Vt = W + S::Vt;
    const T* skd = W + S::C;
    const T* skw = W + S::C + 6 * N;
    const T* skww = W + S::C + 12 * N;
    const T* cO = W + S::C + 18 * N;
    const T* eO = cO + 6;
    const T* vO = cO + 12;
    // ---- edges: primary part, straight to the skeleton
#pragma unroll
    for (int r = lane; r < 12 * N; r += 32) {
      const int slot = r / N, l = r - slot * N, grp = slot >> 2, s1 = slot & 1, s2 = (slot >> 1) & 1;
      T out = __ldg(cb + co.ediag + r) * Ed[r];
      const T *k1, *k2, *f1, *f2;
      int st1, st2;
      T va, vb;
      if (grp == 0) {
        va = Vt[2 * s1 + 4 * s2];
        vb = Vt[1 + 2 * s1 + 4 * s2];
        k1 = skw + (2 + s1) * N; f1 = F + (4 + s2) * N2 + l; st1 = N;
        k2 = skw + (4 + s2) * N; f2 = F + (2 + s1) * N2 + l; st2 = N;
        out = fma(eO[2 + s1], Ed[((1 - s1) + 2 * s2) * N + l], out);
        out = fma(eO[4 + s2], Ed[(s1 + 2 * (1 - s2)) * N + l], out);
      } else if (grp == 1) {
        va = Vt[s1 + 4 * s2];
        vb = Vt[s1 + 2 + 4 * s2];
        k1 = skw + s1 * N; f1 = F + (4 + s2) * N2 + l * N; st1 = 1;
        k2 = skw + (4 + s2) * N; f2 = F + s1 * N2 + l; st2 = N;
        out = fma(eO[s1], Ed[(4 + (1 - s1) + 2 * s2) * N + l], out);
        out = fma(eO[4 + s2], Ed[(4 + s1 + 2 * (1 - s2)) * N + l], out);
      } else {
        va = Vt[s1 + 2 * s2];
        vb = Vt[s1 + 2 * s2 + 4];
        k1 = skw + s1 * N; f1 = F + (2 + s2) * N2 + l * N; st1 = 1;
        k2 = skw + (2 + s2) * N; f2 = F + s1 * N2 + l * N; st2 = 1;
        out = fma(eO[s1], Ed[(8 + (1 - s1) + 2 * s2) * N + l], out);
        out = fma(eO[2 + s2], Ed[(8 + s1 + 2 * (1 - s2)) * N + l], out);
      }
      out = fma(skww[2 * grp * N + l], va, out);
      out = fma(skww[(2 * grp + 1) * N + l], vb, out);
#pragma unroll
      for (int m = 0; m < N; ++m) out = fma(k1[m], f1[m * st1], out);
#pragma unroll
      for (int m = 0; m < N; ++m) out = fma(k2[m], f2[m * st2], out);
      const int off = H[6 + slot];
      if (off >= 0) {
        atomicAdd(v + off + l, out);
        dot = fma(Ed[r], out, dot);
      }
    }
    // ---- vertices
    if (lane < 8) {
      const int slot = lane, sa = slot & 1, sb = (slot >> 1) & 1, sc = slot >> 2;
      T out = __ldg(cb + co.vdiag + slot) * Vt[slot];
      const T* ka = skww + sa * N;
      const T* kb = skww + (2 + sb) * N;
      const T* kc = skww + (4 + sc) * N;
      const T* exl = Ed + (sb + 2 * sc) * N;
      const T* eyl = Ed + (4 + sa + 2 * sc) * N;
      const T* ezl = Ed + (8 + sa + 2 * sb) * N;
#pragma unroll
      for (int m = 0; m < N; ++m) {
        out = fma(ka[m], exl[m], out);
        out = fma(kb[m], eyl[m], out);
        out = fma(kc[m], ezl[m], out);
      }
      out = fma(vO[sa], Vt[slot ^ 1], out);
      out = fma(vO[2 + sb], Vt[slot ^ 2], out);
      out = fma(vO[4 + sc], Vt[slot ^ 4], out);
      const int off = H[18 + slot];
      if (off >= 0) {
        atomicAdd(v + off, out);
        dot = fma(Vt[slot], out, dot);
      }
    }
    // ---- cube columns: expansion, -D^-1, b/t contraction and the z-face
    //      primary part (Table 2; Eq. east_east_primary_part_transformed)
#pragma unroll
    for (int ji = lane; ji < N2; ji += 32) {
      const int j = ji / N, i = ji - j * N;
      const T ai = skd[i], bi = skd[N + i], cj = skd[2 * N + j], dj = skd[3 * N + j];
      const T fb = F[4 * N2 + ji], ft = F[5 * N2 + ji];
      T sb = T(0), stt = T(0);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const Two<T> ez = P2[2 * N + k];
        T x = ai * F[k * N + j];
        x = fma(bi, F[N2 + k * N + j], x);
        x = fma(cj, F[2 * N2 + k * N + i], x);
        x = fma(dj, F[3 * N2 + k * N + i], x);
        x = fma(ez.x, fb, x);
        x = fma(ez.y, ft, x);
        const T vv = __ldg(cb + co.ndinv + k * N2 + ji) * x;
        W[S::cube + (k * N + j) * RS + i] = vv;
        sb = fma(ez.x, vv, sb);
        stt = fma(ez.y, vv, stt);
      }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const T own = s ? ft : fb, opp = s ? fb : ft;
        T pr = ai * Ed[(4 + 2 * s) * N + j];
        pr = fma(bi, Ed[(5 + 2 * s) * N + j], pr);
        pr = fma(cj, Ed[2 * s * N + i], pr);
        pr = fma(dj, Ed[(1 + 2 * s) * N + i], pr);
        T out = fma(__ldg(cb + co.fdiag + (4 + s) * N2 + ji), own, (s ? stt : sb));
        out = fma(cO[4 + s], opp, out);
        out = fma(w0, pr, out);
        const int off = H[4 + s];
        if (off >= 0) {
          atomicAdd(v + off + ji, out);
          dot = fma(own, out, dot);
        }
      }
    }
    __syncwarp();
    // ---- x-faces (k, j = m) and y-faces (k, i = m): primary part and the
    //      w/e and s/n contractions
#pragma unroll
    for (int q = lane; q < N2; q += 32) {
      const int k = q / N, m = q - k * N;
      const Two<T> pa = P2[m], pb = P2[N + m], pc = P2[2 * N + k];   // (skd[m], skd[N+m]), ...
      const T* row = W + S::cube + (k * N + m) * RS;                   // over i
      const T* col = W + S::cube + k * N * RS + m;                     // over j (stride RS)
      T sx0 = T(0), sx1 = T(0), sy0 = T(0), sy1 = T(0);
#pragma unroll
      for (int t = 0; t < N; ++t) {
        const T c = row[t], d = col[t * RS];
        const Two<T> ka = P2[t], kb = P2[N + t];
        sx0 = fma(ka.x, c, sx0);
        sx1 = fma(ka.y, c, sx1);
        sy0 = fma(kb.x, d, sy0);
        sy1 = fma(kb.y, d, sy1);
      }
      const T fx0 = F[q], fx1 = F[N2 + q], fy0 = F[2 * N2 + q], fy1 = F[3 * N2 + q];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        // x-face side s at (k, j = m)
        T pr = pb.x * Ed[(8 + s) * N + k];
        pr = fma(pb.y, Ed[(10 + s) * N + k], pr);
        pr = fma(pc.x, Ed[(4 + s) * N + m], pr);
        pr = fma(pc.y, Ed[(6 + s) * N + m], pr);
        const T own = s ? fx1 : fx0, opp = s ? fx0 : fx1;
        T out = fma(__ldg(cb + co.fdiag + s * N2 + q), own, s ? sx1 : sx0);
        out = fma(cO[s], opp, out);
        out = fma(w0, pr, out);
        int off = H[s];
        if (off >= 0) {
          atomicAdd(v + off + q, out);
          dot = fma(own, out, dot);
        }
        // y-face side s at (k, i = m)
        pr = pa.x * Ed[(8 + 2 * s) * N + k];
        pr = fma(pa.y, Ed[(9 + 2 * s) * N + k], pr);
        pr = fma(pc.x, Ed[s * N + m], pr);
        pr = fma(pc.y, Ed[(2 + s) * N + m], pr);
        const T owny = s ? fy1 : fy0, oppy = s ? fy0 : fy1;
        out = fma(__ldg(cb + co.fdiag + (2 + s) * N2 + q), owny, s ? sy1 : sy0);
        out = fma(cO[2 + s], oppy, out);
        out = fma(w0, pr, out);
        off = H[2 + s];
        if (off >= 0) {
          atomicAdd(v + off + q, out);
          dot = fma(owny, out, dot);
        }
      }
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

// ---------------------------------------------------------------------------
// Thread-per-element variant for p = 2 (n = 1)
// ---------------------------------------------------------------------------
// With one interior node per element every entity carries one value, and the
// packed skeleton is seven regular arrays with the x index fastest: threads
// take consecutive elements in x, so each of an element's 26 loads and 26
// scatter-adds is one contiguous row across the warp.  A thread holds its
// element's boundary values and outputs in registers; the entity offsets come
// from the affine per-slot table, and the class coefficient block (the
// formulas of k_class_coeffs with n = 1) from the transposed per-class table,
// where the consecutive classes of an x-graded row make each coefficient one
// coalesced load (one broadcast load on a uniform mesh).
constexpr int kThreadsP2 = 128;

template <typename T>
__global__ void __launch_bounds__(kThreadsP2, sizeof(T) == 8 ? 3 : 4)
k_tpt_apply_p2(SemGeom g, SemClassTables<T> tab, const T* __restrict__ u, T* __restrict__ v,
               double* __restrict__ partials, PcgState* st, T* __restrict__ ev) {
  __shared__ EntityAffine ent[26];
  if (st != nullptr && st->done) return;
  if (threadIdx.x < 26) entity_affine(g, threadIdx.x, &ent[threadIdx.x]);
  __syncthreads();
  const CoefOffsets co = coef_offsets(1);
  const int nc = tab.ncls, mx = g.mx, my = g.my, mxy = mx * my;
  T dot = T(0);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < (int)g.nelem; e += gridDim.x * blockDim.x) {
    const int ez = e / mxy, rem = e - ez * mxy, ey = rem / mx, ex = rem - ey * mx;
    const int bits = (ex == 0) | ((ex == mx - 1) << 1) | ((ey == 0) << 2) | ((ey == my - 1) << 3) |
                     ((ez == 0) << 4) | ((ez == g.mz - 1) << 5);
    int off[26];
#pragma unroll
    for (int r = 0; r < 26; ++r) {
      const EntityAffine a = ent[r];
      off[r] = entity_offset(a, r, bits, ex, ey, ez, g);
    }
    T F[6], Ed[12], Vt[8];
#pragma unroll
    for (int r = 0; r < 6; ++r) F[r] = off[r] >= 0 ? u[off[r]] : T(0);
#pragma unroll
    for (int r = 0; r < 12; ++r) Ed[r] = off[6 + r] >= 0 ? u[off[6 + r]] : T(0);
#pragma unroll
    for (int r = 0; r < 8; ++r) Vt[r] = off[18 + r] >= 0 ? u[off[18 + r]] : T(0);
    // the class block: d_{dir+1} k_s (skd), scaled by w0 (skw) and w0^2 (skww);
    // d_{dir+1} K_{s,1-s} (cO, eO = w0 cO, vO = w0^2 cO); the diagonals; -D^-1
    const T* cb = tab.coef_soa + elem_class(g, tab, ex, ey, ez);
    auto C = [&](int r) { return __ldg(cb + r * nc); };
    T skd[6], skw[6], skww[6], cO[6], eO[6], vO[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      skd[k] = C(k);
      skw[k] = C(6 + k);
      skww[k] = C(12 + k);
      cO[k] = C(18 + k);
      eO[k] = C(24 + k);
      vO[k] = C(30 + k);
    }
    // condensed part: one eigenspace value
    T x = skd[0] * F[0];
#pragma unroll
    for (int k = 1; k < 6; ++k) x = fma(skd[k], F[k], x);
    const T vv = C(co.ndinv) * x;
    T Fo[6], Eo[12], Vo[8];
    // faces: primary part + condensed contraction
#pragma unroll
    for (int slot = 0; slot < 6; ++slot) {
      const int dd = slot >> 1, s = slot & 1;
      T out = fma(C(co.fdiag + slot), F[slot], skd[slot] * vv);
      out = fma(cO[slot], F[slot ^ 1], out);
      if (dd == 0) {
        out = fma(skw[2], Ed[8 + s], out);
        out = fma(skw[3], Ed[10 + s], out);
        out = fma(skw[4], Ed[4 + s], out);
        out = fma(skw[5], Ed[6 + s], out);
      } else if (dd == 1) {
        out = fma(skw[0], Ed[8 + 2 * s], out);
        out = fma(skw[1], Ed[9 + 2 * s], out);
        out = fma(skw[4], Ed[s], out);
        out = fma(skw[5], Ed[2 + s], out);
      } else {
        out = fma(skw[0], Ed[4 + 2 * s], out);
        out = fma(skw[1], Ed[5 + 2 * s], out);
        out = fma(skw[2], Ed[2 * s], out);
        out = fma(skw[3], Ed[1 + 2 * s], out);
      }
      Fo[slot] = out;
    }
    // edges: diagonal, the two vertices, the two faces, the two parallel edges
#pragma unroll
    for (int slot = 0; slot < 12; ++slot) {
      const int grp = slot >> 2, s1 = slot & 1, s2 = (slot >> 1) & 1;
      T out = C(co.ediag + slot) * Ed[slot];
      if (grp == 0) {
        out = fma(skww[0], Vt[2 * s1 + 4 * s2], out);
        out = fma(skww[1], Vt[1 + 2 * s1 + 4 * s2], out);
        out = fma(skw[2 + s1], F[4 + s2], out);
        out = fma(skw[4 + s2], F[2 + s1], out);
        out = fma(eO[2 + s1], Ed[(1 - s1) + 2 * s2], out);
        out = fma(eO[4 + s2], Ed[s1 + 2 * (1 - s2)], out);
      } else if (grp == 1) {
        out = fma(skww[2], Vt[s1 + 4 * s2], out);
        out = fma(skww[3], Vt[s1 + 2 + 4 * s2], out);
        out = fma(skw[s1], F[4 + s2], out);
        out = fma(skw[4 + s2], F[s1], out);
        out = fma(eO[s1], Ed[4 + (1 - s1) + 2 * s2], out);
        out = fma(eO[4 + s2], Ed[4 + s1 + 2 * (1 - s2)], out);
      } else {
        out = fma(skww[4], Vt[s1 + 2 * s2], out);
        out = fma(skww[5], Vt[s1 + 2 * s2 + 4], out);
        out = fma(skw[s1], F[2 + s2], out);
        out = fma(skw[2 + s2], F[s1], out);
        out = fma(eO[s1], Ed[8 + (1 - s1) + 2 * s2], out);
        out = fma(eO[2 + s2], Ed[8 + s1 + 2 * (1 - s2)], out);
      }
      Eo[slot] = out;
    }
    // vertices: diagonal, the three edges, the three neighbouring vertices
#pragma unroll
    for (int slot = 0; slot < 8; ++slot) {
      const int sa = slot & 1, sb = (slot >> 1) & 1, sc = slot >> 2;
      T out = C(co.vdiag + slot) * Vt[slot];
      out = fma(skww[sa], Ed[sb + 2 * sc], out);
      out = fma(skww[2 + sb], Ed[4 + sa + 2 * sc], out);
      out = fma(skww[4 + sc], Ed[8 + sa + 2 * sb], out);
      out = fma(vO[sa], Vt[slot ^ 1], out);
      out = fma(vO[2 + sb], Vt[slot ^ 2], out);
      out = fma(vO[4 + sc], Vt[slot ^ 4], out);
      Vo[slot] = out;
    }
    // scatter R and the element share of x^T (A x)
#pragma unroll
    for (int r = 0; r < 6; ++r)
      if (off[r] >= 0) { atomicAdd(v + off[r], Fo[r]); dot = fma(F[r], Fo[r], dot); }
#pragma unroll
    for (int r = 0; r < 12; ++r)
      if (off[6 + r] >= 0) {
        if (ev != nullptr) ev[(long long)r * g.nelem + e] = Eo[r];   // fixed-order mode: summed by k_ev_sum
        else atomicAdd(v + off[6 + r], Eo[r]);
        dot = fma(Ed[r], Eo[r], dot);
      }
#pragma unroll
    for (int r = 0; r < 8; ++r)
      if (off[18 + r] >= 0) {
        if (ev != nullptr) ev[(12LL + r) * g.nelem + e] = Vo[r];
        else atomicAdd(v + off[18 + r], Vo[r]);
        dot = fma(Vt[r], Vo[r], dot);
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

template <typename T>
__global__ void k_coef_soa(const T* __restrict__ coef, T* __restrict__ soa, int ncls, int stride) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)ncls * stride;
       t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / stride), r = (int)(t - (long long)c * stride);
    soa[(long long)r * ncls + c] = coef[t];
  }
}

template <typename T>
void launch_p2(const SemGeom& g, const SemClassTables<T>& t, const T* x, T* y, double* partials, PcgState* st,
               cudaStream_t s, T* ev = nullptr) {
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tpt_apply_p2<T>, kThreadsP2, 0);
  if (occ < 1) occ = 1;
  long long grid = (long long)num_sms_cached() * occ;
  const long long need = (g.nelem + kThreadsP2 - 1) / kThreadsP2;
  if (grid > need) grid = need;
  k_tpt_apply_p2<T><<<(int)grid, kThreadsP2, 0, s>>>(g, t, x, y, partials, st, ev);
  sem_count_launch();
}

template <typename T, int N>
size_t warp_smem(int wpb) {
  return ((size_t)wpb * kWarpHdr * 4 + 31) / 32 * 32 + (size_t)wpb * WarpSm<N>::size * sizeof(T);
}

template <typename T, int N>
void launch_warp(const SemGeom& g, const SemClassTables<T>& t, const T* x, T* y, double* partials, PcgState* st,
                 double w0, cudaStream_t s) {
  const int wpb = kThreads / 32;
  const size_t smem = warp_smem<T, N>(wpb);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tpt_apply_warp<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tpt_apply_warp<T, N>, kThreads, smem);
  if (occ < 1) occ = 1;
  long long grid = (long long)num_sms_cached() * occ;
  const long long need = (g.nelem + wpb - 1) / wpb;
  if (grid > need) grid = need;
  k_tpt_apply_warp<T, N><<<(int)grid, kThreads, smem, s>>>(g, t, x, y, partials, st, (T)w0);
  sem_count_launch();
}

template <typename T, int NC>
void launch_nc(const SemGeom& g, const SemClassTables<T>& t, const T* x, T* y, double* partials, PcgState* st,
               const ApplyConfig& c, cudaStream_t s, T* ev = nullptr) {
  static bool attr = false;
  if (!attr) {   // once per instantiation; the first launch happens in sem_setup, outside any capture
    cudaFuncSetAttribute(k_tpt_apply<T, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  int o = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_tpt_apply<T, NC>, c.threads, c.smem);
  if (o < 1) o = 1;
  const long long ntiles = (g.nelem + c.epb - 1) / c.epb;
  long long grid = (long long)num_sms_cached() * o;
  if (grid > ntiles) grid = ntiles;
  k_tpt_apply<T, NC><<<(int)grid, c.threads, c.smem, s>>>(g, t, x, y, c.epb, c.ks, partials, st, ev);
  sem_count_launch();
}

}  // namespace

ApplyConfig sem_apply_config(int n, size_t elem_bytes) {
  ApplyConfig c;
  c.kind = kApplyCta;
  c.threads = kThreads;
  const size_t big = 200 * 1024, small = 96 * 1024;
  int ks = n;
  int epb = 1;
  // one thread per (j, i) cube column: aim for epb * n^2 close to the block size
  const int n2 = n * n;
  const int want = n2 >= kThreads ? 1 : kThreads / n2;
  epb = want > 64 ? 64 : want;
  auto bytes = [&](int e, int k) { return hdr_bytes(e) + (size_t)e * elem_sm(n, k).size * elem_bytes; };
  while (epb > 1 && bytes(epb, ks) > small) --epb;
  while (ks > 1 && bytes(epb, ks) > (epb == 1 ? big : small)) ks = (ks + 1) / 2;
  c.epb = epb;
  c.ks = ks;
  c.smem = bytes(epb, ks);
  return c;
}

ApplyConfig sem_apply_config_make(int n, size_t elem_bytes, int epb, int ks) {
  ApplyConfig c;
  c.kind = kApplyCta;
  c.threads = kThreads;
  c.epb = epb;
  c.ks = ks;
  c.smem = (epb >= 1 && ks >= 1) ? hdr_bytes(epb) + (size_t)epb * elem_sm(n, ks).size * elem_bytes : 0;
  return c;
}

ApplyConfig sem_apply_config_kind(int kind) {
  ApplyConfig c;
  c.kind = kind;
  return c;
}

bool sem_apply_config_valid(int n, size_t elem_bytes, const ApplyConfig& c) {
  switch (c.kind) {
    case kApplyAuto:
      return true;
    case kApplyCta: {
      if (c.epb < 1 || c.epb > 64 || c.ks < 1 || c.ks > n || c.threads != kThreads) return false;
      const size_t need = hdr_bytes(c.epb) + (size_t)c.epb * elem_sm(n, c.ks).size * elem_bytes;
      return need == c.smem && need <= 200 * 1024;
    }
    case kApplyWarp:
      return elem_bytes == 4 && n >= 3 && n <= 7;
    case kApplyPlane:
      return elem_bytes == 4 && plane_supported(n);
    case kApplyElement:
      return n == 1 || (elem_bytes == 4 && elem_supported(n));
    case kApplySlab:
      return elem_bytes == 4 && slab_supported(n);
    case kApplyRow:
      return elem_bytes == 4 && row_supported(n);
    case kApplyPencil:
      return elem_bytes == 4 && pencil_supported(n);
    default:
      return false;
  }
}

// Measured on GB300: FP64 is bound by the FP64 pipe and runs best with the
// CTA tile; FP32 at 3 <= n <= 15 with the plane kernels and at 16 <= n <= 31
// with the k-slab kernel; n = 1, and n = 2 in FP32, with one thread per
// element (at n = 3 its 254 registers leave too few warps: 150 against the
// plane kernel's 125 us at p = 4).
// Position of element (ex, ey, ez) in the visiting order of elem_visit.
__device__ __forceinline__ long long elem_visit_index(const SemGeom& g, int ex, int ey, int ez) {
  if (g.slow == 0) return (long long)ex * g.my * g.mz + (long long)ez * g.my + ey;
  if (g.slow == 1) return (long long)ey * g.mx * g.mz + (long long)ez * g.mx + ex;
  return ex + (long long)g.mx * (ey + (long long)g.my * ez);
}

// Fixed-order assembly of the edge and vertex outputs (the R^T of Sec. 4 for
// the entities shared by four and eight elements).  ev holds each element's
// contributions, (12 n + 8) values per element (edge slot q at position
// q n + l, vertex slot r at 12 n + r): visit != 0, element-major at the
// element's visit position (the CTA tile writes an element's values
// together); visit == 0, position-major over the x-fastest element index (the
// one-thread-per-element kernel writes coalesced).  Every entity off the
// Dirichlet boundary has all
// its neighbours; it is summed by the one that sees it at its upper sides
// (edge slots 3, 7, 11, vertex slot 7), in the order of the side bits, and
// added to v: the result does not depend on the order the elements ran in.
template <typename T>
__global__ void k_ev_sum(SemGeom g, const T* __restrict__ ev, T* __restrict__ v, int visit, const PcgState* st) {
  if (st != nullptr && st->done) return;   // the operator launch before it did not run (stopped CG, closed gate)
  // 32-bit index arithmetic (nelem (3 n + 1) < 2^31 whenever N_B is); the
  // thread order follows the layout so that neighbouring threads read
  // neighbouring values: position fastest for the element-major layout,
  // element fastest for the position-major one
  const int n = g.n, per = 3 * n + 1, ne_all = (int)g.nelem, mx = g.mx, my = g.my;
  const int stride = 12 * n + 8;
  const int total = ne_all * per;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int e, r;
    if (visit) { e = t / per; r = t - e * per; }
    else { r = t / ne_all; e = t - r * ne_all; }
    const int ez = e / (mx * my), rem = e - ez * (mx * my), ey = rem / mx, ex = rem - ey * mx;
    bool dir;
    T sum = T(0);
    if (r < 3 * n) {
      const int grp = r / n, l = r - grp * n;
      const long long off = edge_base(g, ex, ey, ez, 4 * grp + 3, &dir);
      if (dir) continue;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int s1 = q & 1, s2 = q >> 1;
        int nx = ex, ny = ey, nz = ez;
        if (grp == 0) { ny += 1 - s1; nz += 1 - s2; }
        else if (grp == 1) { nx += 1 - s1; nz += 1 - s2; }
        else { nx += 1 - s1; ny += 1 - s2; }
        const int pos = (4 * grp + q) * n + l;
        sum += visit ? ev[elem_visit_index(g, nx, ny, nz) * stride + pos]
                     : ev[(long long)pos * ne_all + nx + mx * (ny + my * nz)];
      }
      v[off + l] += sum;
    } else {
      const long long off = vert_index(g, ex, ey, ez, 7, &dir);
      if (dir) continue;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int nx = ex + 1 - (q & 1), ny = ey + 1 - ((q >> 1) & 1), nz = ez + 1 - (q >> 2);
        const int pos = 12 * n + q;
        sum += visit ? ev[elem_visit_index(g, nx, ny, nz) * stride + pos]
                     : ev[(long long)pos * ne_all + nx + mx * (ny + my * nz)];
      }
      v[off] += sum;
    }
  }
}

template <typename T>
void launch_ev_sum(const SemGeom& g, const T* ev, T* v, int visit, const PcgState* st, cudaStream_t s) {
  const long long work = g.nelem * (3LL * g.n + 1);
  long long blocks = (work + 255) / 256;
  if (blocks > (long long)num_sms_cached() * 16) blocks = (long long)num_sms_cached() * 16;
  if (blocks < 1) blocks = 1;
  k_ev_sum<T><<<(int)blocks, 256, 0, s>>>(g, ev, v, visit, st);
  sem_count_launch();
}

int sem_apply_default_kind(int n, size_t elem_bytes) {
  if (n == 1 || (elem_bytes == 4 && n == 2)) return kApplyElement;
  if (elem_bytes == 4 && plane_supported(n)) return kApplyPlane;
  if (elem_bytes == 4 && slab_supported(n)) return kApplySlab;
  return kApplyCta;
}

template <typename T>
void launch_tpt_apply(const SemGeom& g, const SemBasis& b, const SemClassTables<T>& t, const T* x, T* y,
                      double* partials, PcgState* st, cudaStream_t s, const ApplyConfig* cfg) {
  const bool explicit_cfg = cfg != nullptr && cfg->kind != kApplyAuto && sem_apply_config_valid(g.n, sizeof(T), *cfg);
  int kind = explicit_cfg ? cfg->kind : sem_apply_default_kind(g.n, sizeof(T));
  if constexpr (sizeof(T) == 4) {
    if ((kind == kApplyPlane || kind == kApplySlab) && t.plane == nullptr) kind = kApplyCta;   // tables not built (cannot happen via the API)
    if (kind == kApplyPencil && t.plane != nullptr) {
      launch_pencil_apply(g, t, x, y, partials, st, s);
      return;
    }
    if (kind == kApplyRow) {
      if (row_usable(g, x, y)) {
        launch_row_apply(g, b, t, x, y, partials, st, s);
        return;
      }
      kind = kApplyPlane;   // too many segments, or x and y differently aligned modulo 16 bytes
    }
    if (kind == kApplyPlane) {
      launch_plane_apply(g, t, x, y, partials, st, s);
      return;
    }
    if (kind == kApplySlab) {
      launch_slab_apply(g, t, x, y, partials, st, s);
      return;
    }
    if (kind == kApplyWarp) {
      switch (g.n) {
        case 3: launch_warp<T, 3>(g, t, x, y, partials, st, b.w0, s); return;
        case 4: launch_warp<T, 4>(g, t, x, y, partials, st, b.w0, s); return;
        case 5: launch_warp<T, 5>(g, t, x, y, partials, st, b.w0, s); return;
        case 6: launch_warp<T, 6>(g, t, x, y, partials, st, b.w0, s); return;
        default: launch_warp<T, 7>(g, t, x, y, partials, st, b.w0, s); return;
      }
    }
  }
  // fixed-order edge and vertex sums: the CTA tile (or, at n = 1, the
  // element kernel) writes each element's shares to ev, k_ev_sum adds them
  T* ev = cfg != nullptr ? static_cast<T*>(cfg->ev) : nullptr;
  if (ev != nullptr) {
    if (g.n == 1) {
      launch_p2<T>(g, t, x, y, partials, st, s, ev);
      launch_ev_sum<T>(g, ev, y, 0, st, s);
      return;
    }
    kind = kApplyCta;
  }
  if (kind == kApplyElement) {
    if constexpr (sizeof(T) == 4) {
      if (g.n != 1) {
        if (t.plane_soa != nullptr) {
          launch_elem_apply(g, t, x, y, partials, st, s);
          return;
        }
        kind = kApplyCta;   // tables not built (cannot happen via the API)
      }
    }
    if (kind == kApplyElement) {
      launch_p2<T>(g, t, x, y, partials, st, s);
      return;
    }
  }
  const ApplyConfig c = (explicit_cfg && cfg->kind == kApplyCta) ? *cfg : sem_apply_config(g.n, sizeof(T));
  if (ev != nullptr) {
    switch (g.n) {
      case 3: launch_nc<T, 3>(g, t, x, y, partials, st, c, s, ev); break;
      case 7: launch_nc<T, 7>(g, t, x, y, partials, st, c, s, ev); break;
      case 15: launch_nc<T, 15>(g, t, x, y, partials, st, c, s, ev); break;
      case 31: launch_nc<T, 31>(g, t, x, y, partials, st, c, s, ev); break;
      default: launch_nc<T, 0>(g, t, x, y, partials, st, c, s, ev); break;
    }
    launch_ev_sum<T>(g, ev, y, 1, st, s);
    return;
  }
  switch (g.n) {
    case 1: launch_nc<T, 1>(g, t, x, y, partials, st, c, s); break;
    case 3: launch_nc<T, 3>(g, t, x, y, partials, st, c, s); break;
    case 7: launch_nc<T, 7>(g, t, x, y, partials, st, c, s); break;
    case 15: launch_nc<T, 15>(g, t, x, y, partials, st, c, s); break;
    case 31: launch_nc<T, 31>(g, t, x, y, partials, st, c, s); break;
    default: launch_nc<T, 0>(g, t, x, y, partials, st, c, s); break;
  }
}

template <typename T>
void launch_class_coeffs(const SemGeom& g, const SemBasis& b, const double* dcoef, const double* dinv, T* coef,
                         cudaStream_t s) {
  const long long work = (long long)g.ux * g.uy * g.uz * coef_offsets(g.n).stride;
  long long blocks = (work + 255) / 256;
  if (blocks > (long long)num_sms_cached() * 16) blocks = (long long)num_sms_cached() * 16;
  if (blocks < 1) blocks = 1;
  k_class_coeffs<T><<<(int)blocks, 256, 0, s>>>(g, b, dcoef, dinv, coef);
  sem_count_launch();
}

template void launch_tpt_apply<double>(const SemGeom&, const SemBasis&, const SemClassTables<double>&,
                                       const double*, double*, double*, PcgState*, cudaStream_t,
                                       const ApplyConfig*);
template void launch_tpt_apply<float>(const SemGeom&, const SemBasis&, const SemClassTables<float>&,
                                      const float*, float*, double*, PcgState*, cudaStream_t, const ApplyConfig*);
template <typename T>
void launch_coef_soa(const SemGeom& g, const T* coef, T* soa, long long stride_ll, cudaStream_t s) {
  const int ncls = g.ux * g.uy * g.uz, stride = (int)stride_ll;
  long long blocks = ((long long)ncls * stride + 255) / 256;
  if (blocks > (long long)num_sms_cached() * 16) blocks = (long long)num_sms_cached() * 16;
  if (blocks < 1) blocks = 1;
  k_coef_soa<T><<<(int)blocks, 256, 0, s>>>(coef, soa, ncls, stride);
  sem_count_launch();
}

template void launch_coef_soa<double>(const SemGeom&, const double*, double*, long long, cudaStream_t);
template void launch_coef_soa<float>(const SemGeom&, const float*, float*, long long, cudaStream_t);
template void launch_class_coeffs<double>(const SemGeom&, const SemBasis&, const double*, const double*, double*,
                                          cudaStream_t);
template void launch_class_coeffs<float>(const SemGeom&, const SemBasis&, const double*, const double*, float*,
                                         cudaStream_t);

SEM_DEBUG_TU(apply)
