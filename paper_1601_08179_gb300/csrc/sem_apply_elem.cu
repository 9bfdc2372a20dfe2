// Thread-per-element variant of the transformed condensed operator (Sec. 6 of
// the paper) for FP32 and n = 2, 3 (p = 3, 4): the inner operator of the
// mixed-precision solve at low degree.
//
// The element operator is the one of the other variants (sem_apply.cu,
// sem_apply_plane.cu): the six faces expanded into the interior eigenspace
// (Table 2), D^-1 (Eq. hii_diagonal), the contraction back onto the faces,
// and the primary part H~_BB restricted to the skeleton.  At these degrees an
// element's 6 n^2 + 12 n + 8 boundary values (98 at n = 3), its n^3
// eigenspace points and the six contractions fit in one thread's registers,
// so no lane exchanges data with another:
// * elements are visited x fastest, so each of an element's gathers and
//   scatter-adds is one row across the warp with a stride of one entity;
// * the entity offsets come from the affine per-slot table, the class
//   coefficients (the block of plane_layout(n)) from its transposed copy,
//   where the consecutive classes of an x-graded row make each coefficient
//   one coalesced load;
// * D^-1 = 1 / (d0 + d1 lambda_i + d2 lambda_j + d3 lambda_k) is formed per
//   point with one reciprocal, as in the plane kernels.
#include <cuda_runtime.h>

#include "sem_device.cuh"
#include "sem_kernels.cuh"

using namespace semdev;

namespace {

constexpr int kElemThreads = 128;

template <int N>
__global__ void __launch_bounds__(kElemThreads, 2)
k_tpt_apply_elem(SemGeom g, SemClassTables<float> tab, const float* __restrict__ u, float* __restrict__ v,
                 double* __restrict__ partials, PcgState* st) {
  __shared__ EntityAffine ent[26];
  if (st != nullptr && st->done) return;
  if (threadIdx.x < 26) entity_affine(g, threadIdx.x, &ent[threadIdx.x]);
  __syncthreads();
  constexpr int N2 = N * N;
  const PlaneLayout L = plane_layout(N);
  const int nc = tab.ncls, mx = g.mx, my = g.my, mxy = mx * my;
  float dot = 0.f;
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
    // gather R^T: faces F[slot][slow * N + fast] (x-faces (k, j), y-faces
    // (k, i), z-faces (j, i)); edges E[q][l] (x-edges q = sb + 2 sc, y-edges
    // 4 + sa + 2 sc, z-edges 8 + sa + 2 sb); vertices Vt[sa + 2 sb + 4 sc]
    float F[6][N2], E[12][N], Vt[8];
#pragma unroll
    for (int s = 0; s < 6; ++s)
#pragma unroll
      for (int t = 0; t < N2; ++t) F[s][t] = off[s] >= 0 ? u[off[s] + t] : 0.f;
#pragma unroll
    for (int q = 0; q < 12; ++q)
#pragma unroll
      for (int l = 0; l < N; ++l) E[q][l] = off[6 + q] >= 0 ? u[off[6 + q] + l] : 0.f;
#pragma unroll
    for (int r = 0; r < 8; ++r) Vt[r] = off[18 + r] >= 0 ? u[off[18 + r]] : 0.f;
    // class coefficients: entry r of class c at r * nc + c
    const float* cb = tab.plane_soa + elem_class(g, tab, ex, ey, ez);
    auto C = [&](int r) { return __ldg(cb + r * nc); };
    float a[N], b[N], l1[N], l2[N], l3[N], cc[N], dd[N], ee[N], gg[N];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      a[m] = C(L.pa + m);
      b[m] = C(L.pb + m);
      l1[m] = C(L.pl1 + m);
      l2[m] = C(L.pl2 + m);
      l3[m] = C(L.pl3 + m);
      cc[m] = C(L.pq + 4 * m);
      dd[m] = C(L.pq + 4 * m + 1);
      ee[m] = C(L.pq + 4 * m + 2);
      gg[m] = C(L.pq + 4 * m + 3);
    }
    float cO[6], fc[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      cO[q] = C(L.ps + q);
      fc[q] = C(L.ps + 6 + q);
    }
    const float w0 = C(L.ps + 32), w02 = C(L.ps + 33), d0 = C(L.ps + 34);

    // ---- condensed part: expansion, D^-1, the six contractions
    float Xo[2][N2], Yo[2][N2], Zo[2][N2];
#pragma unroll
    for (int t = 0; t < N2; ++t) Xo[0][t] = Xo[1][t] = Yo[0][t] = Yo[1][t] = Zo[0][t] = Zo[1][t] = 0.f;
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
      for (int j = 0; j < N; ++j)
#pragma unroll
        for (int i = 0; i < N; ++i) {
          float x = a[i] * F[0][k * N + j];
          x = fmaf(b[i], F[1][k * N + j], x);
          x = fmaf(cc[j], F[2][k * N + i], x);
          x = fmaf(dd[j], F[3][k * N + i], x);
          x = fmaf(ee[k], F[4][j * N + i], x);
          x = fmaf(gg[k], F[5][j * N + i], x);
          const float w = x * rcp_approx(d0 + l1[i] + l2[j] + l3[k]);   // D^-1 x (the sign is applied at the outputs)
          Xo[0][k * N + j] = fmaf(a[i], w, Xo[0][k * N + j]);
          Xo[1][k * N + j] = fmaf(b[i], w, Xo[1][k * N + j]);
          Yo[0][k * N + i] = fmaf(cc[j], w, Yo[0][k * N + i]);
          Yo[1][k * N + i] = fmaf(dd[j], w, Yo[1][k * N + i]);
          Zo[0][j * N + i] = fmaf(ee[k], w, Zo[0][j * N + i]);
          Zo[1][j * N + i] = fmaf(gg[k], w, Zo[1][j * N + i]);
        }

    // ---- faces: diagonal, opposite face, the four edge lines, minus the
    //      condensed sum; scatter-add and the element share of x^T (A x)
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const int off0 = off[f], off1 = off[2 + f], off2 = off[4 + f];
#pragma unroll
      for (int s = 0; s < N; ++s)      // slow index (k for the x- and y-faces, j for the z-faces)
#pragma unroll
        for (int t = 0; t < N; ++t) {  // fast index (j, i, i)
          {  // x-face f at (k, j) = (s, t)
            const int k = s, j = t;
            float o = (fc[f] + w0 * (l2[j] + l3[k])) * F[f][k * N + j];
            o = fmaf(cO[f], F[1 - f][k * N + j], o);
            o = fmaf(w0, fmaf(cc[j], E[8 + f][k], fmaf(dd[j], E[10 + f][k], fmaf(ee[k], E[4 + f][j], gg[k] * E[6 + f][j]))), o);
            o -= Xo[f][k * N + j];
            if (off0 >= 0) {
              atomicAdd(v + off0 + k * N + j, o);
              dot = fmaf(F[f][k * N + j], o, dot);
            }
          }
          {  // y-face f at (k, i) = (s, t)
            const int k = s, i = t;
            float o = (fc[2 + f] + w0 * (l1[i] + l3[k])) * F[2 + f][k * N + i];
            o = fmaf(cO[2 + f], F[3 - f][k * N + i], o);
            o = fmaf(w0, fmaf(a[i], E[8 + 2 * f][k], fmaf(b[i], E[9 + 2 * f][k], fmaf(ee[k], E[f][i], gg[k] * E[2 + f][i]))), o);
            o -= Yo[f][k * N + i];
            if (off1 >= 0) {
              atomicAdd(v + off1 + k * N + i, o);
              dot = fmaf(F[2 + f][k * N + i], o, dot);
            }
          }
          {  // z-face f at (j, i) = (s, t)
            const int j = s, i = t;
            float o = (fc[4 + f] + w0 * (l1[i] + l2[j])) * F[4 + f][j * N + i];
            o = fmaf(cO[4 + f], F[5 - f][j * N + i], o);
            o = fmaf(w0, fmaf(a[i], E[4 + 2 * f][j], fmaf(b[i], E[5 + 2 * f][j], fmaf(cc[j], E[2 * f][i], dd[j] * E[1 + 2 * f][i]))), o);
            o -= Zo[f][j * N + i];
            if (off2 >= 0) {
              atomicAdd(v + off2 + j * N + i, o);
              dot = fmaf(F[4 + f][j * N + i], o, dot);
            }
          }
        }
    }
    // ---- edges: diagonal, the two vertices, the two face lines, the two
    //      parallel edges
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int s1 = q & 1, s2 = q >> 1;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        {  // x-edge Ex[sb][sc] at i = l
          const int sb = s1, sc = s2;
          float szc = 0.f, sy = 0.f;   // z-face sc column l over j; y-face sb column l over k
#pragma unroll
          for (int m = 0; m < N; ++m) {
            szc = fmaf(sb ? dd[m] : cc[m], F[4 + sc][m * N + l], szc);
            sy = fmaf(sc ? gg[m] : ee[m], F[2 + sb][m * N + l], sy);
          }
          float o = (w02 * (d0 + l1[l]) + C(L.ps + 12 + q)) * E[q][l];
          o = fmaf(w02, fmaf(a[l], Vt[2 * sb + 4 * sc], b[l] * Vt[1 + 2 * sb + 4 * sc]), o);
          o = fmaf(w0, szc + sy, o);
          o = fmaf(w0 * cO[2 + sb], E[(1 - sb) + 2 * sc][l], o);
          o = fmaf(w0 * cO[4 + sc], E[sb + 2 * (1 - sc)][l], o);
          if (off[6 + q] >= 0) {
            atomicAdd(v + off[6 + q] + l, o);
            dot = fmaf(E[q][l], o, dot);
          }
        }
        {  // y-edge Ey[sa][sc] at j = l
          const int sa = s1, sc = s2;
          float szr = 0.f, sx = 0.f;   // z-face sc row l over i; x-face sa column l over k
#pragma unroll
          for (int m = 0; m < N; ++m) {
            szr = fmaf(sa ? b[m] : a[m], F[4 + sc][l * N + m], szr);
            sx = fmaf(sc ? gg[m] : ee[m], F[sa][m * N + l], sx);
          }
          float o = (w02 * (d0 + l2[l]) + C(L.ps + 16 + q)) * E[4 + q][l];
          o = fmaf(w02, fmaf(cc[l], Vt[sa + 4 * sc], dd[l] * Vt[sa + 2 + 4 * sc]), o);
          o = fmaf(w0, szr + sx, o);
          o = fmaf(w0 * cO[sa], E[4 + (1 - sa) + 2 * sc][l], o);
          o = fmaf(w0 * cO[4 + sc], E[4 + sa + 2 * (1 - sc)][l], o);
          if (off[10 + q] >= 0) {
            atomicAdd(v + off[10 + q] + l, o);
            dot = fmaf(E[4 + q][l], o, dot);
          }
        }
        {  // z-edge Ez[sa][sb] at k = l
          const int sa = s1, sb = s2;
          float syr = 0.f, sxr = 0.f;   // y-face sb row l over i; x-face sa row l over j
#pragma unroll
          for (int m = 0; m < N; ++m) {
            syr = fmaf(sa ? b[m] : a[m], F[2 + sb][l * N + m], syr);
            sxr = fmaf(sb ? dd[m] : cc[m], F[sa][l * N + m], sxr);
          }
          float o = (w02 * (d0 + l3[l]) + C(L.ps + 20 + q)) * E[8 + q][l];
          o = fmaf(w02, fmaf(ee[l], Vt[sa + 2 * sb], gg[l] * Vt[sa + 2 * sb + 4]), o);
          o = fmaf(w0, syr + sxr, o);
          o = fmaf(w0 * cO[sa], E[8 + (1 - sa) + 2 * sb][l], o);
          o = fmaf(w0 * cO[2 + sb], E[8 + sa + 2 * (1 - sb)][l], o);
          if (off[14 + q] >= 0) {
            atomicAdd(v + off[14 + q] + l, o);
            dot = fmaf(E[8 + q][l], o, dot);
          }
        }
      }
    }
    // ---- vertices: diagonal, the three edge lines, the three neighbours
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int sa = r & 1, sb = (r >> 1) & 1, sc = r >> 2;
      float sv = 0.f;
#pragma unroll
      for (int m = 0; m < N; ++m) {
        sv = fmaf(sa ? b[m] : a[m], E[sb + 2 * sc][m], sv);
        sv = fmaf(sb ? dd[m] : cc[m], E[4 + sa + 2 * sc][m], sv);
        sv = fmaf(sc ? gg[m] : ee[m], E[8 + sa + 2 * sb][m], sv);
      }
      float o = C(L.ps + 24 + r) * Vt[r];
      o = fmaf(w02, sv, o);
      o = fmaf(w02 * cO[sa], Vt[r ^ 1], o);
      o = fmaf(w02 * cO[2 + sb], Vt[r ^ 2], o);
      o = fmaf(w02 * cO[4 + sc], Vt[r ^ 4], o);
      if (off[18 + r] >= 0) {
        atomicAdd(v + off[18 + r], o);
        dot = fmaf(Vt[r], o, dot);
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

template <int N>
void launch_elem_n(const SemGeom& g, const SemClassTables<float>& t, const float* x, float* y, double* partials,
                   PcgState* st, cudaStream_t s) {
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tpt_apply_elem<N>, kElemThreads, 0);
  if (occ < 1) occ = 1;
  long long grid = (long long)sem_num_sms() * occ;
  const long long need = (g.nelem + kElemThreads - 1) / kElemThreads;
  if (grid > need) grid = need;
  k_tpt_apply_elem<N><<<(int)grid, kElemThreads, 0, s>>>(g, t, x, y, partials, st);
  sem_count_launch();
}

}  // namespace

void launch_elem_apply(const SemGeom& g, const SemClassTables<float>& t, const float* x, float* y,
                       double* partials, PcgState* st, cudaStream_t s) {
  if (g.n == 2) launch_elem_n<2>(g, t, x, y, partials, st, s);
  else launch_elem_n<3>(g, t, x, y, partials, st, s);
}

SEM_DEBUG_TU(elem)
