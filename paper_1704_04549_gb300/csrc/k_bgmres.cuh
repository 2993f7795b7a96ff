// Device code of the per-system batched GMRES (tpp_batch_gmres, host side in
// k_bgmres.cu; one translation unit per lane-group width).
//
// Per-system batched GMRES over batches of isolated elements (block-diagonal
// systems S_e x = b_{e,r}: mass, volume and outflow face terms of one element,
// Sec. 3.4 with the neighbour coupling dropped), every (element, right-hand side)
// system with its own Arnoldi process, Givens rotations, restarts and
// convergence test (Sec. 5 opening: right-preconditioned restarted GMRES with
// the Kronecker preconditioner of Alg. 2d-apply / 3d-apply).
//
// Execution model.  One persistent launch per lane-group width NM (8, 16 or 32
// lanes per system): CTAs pull elements from a queue that holds every element of
// every degree group handled by the launch, most expensive first.  A CTA stages
// the element's factors and flux coefficients in shared memory once; its warps
// then solve the element's right-hand sides, 32 / NM systems per warp, lane i of a
// group owning row i of the n x n matrix of a 2D vector (of each z slice in 3D).
// Krylov vectors live in a per-group slot of global memory (L1 / L2 resident);
// Hessenberg columns and Givens rotations in a per-group scalar slot.
//
// Precision.  FP64: GMRES(m) in FP64 to the relative residual tol.  Mixed: FP64
// iterative refinement (true residual with the FP64 operator) around FP32
// GMRES(m) solves of the correction (FP32 operator, FP32 factors, FP32 Arnoldi
// vectors; Hessenberg and Givens in FP64).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#pragma once
#include "tpp_internal.cuh"

namespace tpp {
namespace bg {

// the element data one CTA stages (pointers into the group's context)
template <typename T>
struct GroupData {
  const T *cx, *cy, *cz, *fa;                  // flux coefficients (dt folded in)
  const T *SA, *SB, *Q1, *Q2, *T1, *T2, *Azi;  // two-sided factors (3D: of D1, and Azi)
};

struct BGroup {
  int dim, n, R, nloc;
  int64_t E;
  double hd;                  // h^d
  const Tables* T;
  const uint32_t* masks;      // 2x2-block structure of T1 / T2
  GroupData<double> d64;
  GroupData<float> d32;       // FP32 copies (mixed precision; NULL otherwise)
  const double* b;
  double* x;
  int32_t* iters;             // per system (optional)
  double* relres;             // per system (optional)
};

// device-side totals of one batched solve
struct BatchStats {
  unsigned long long total_iters;   // Arnoldi steps summed over the systems
  int32_t max_iters, unconverged, outer_max, pad;
  double max_relres;                // largest final true relative residual
};

// one work item: right-hand sides [r0, r0 + lane groups of a CTA) of one element
struct BItem {
  int32_t group, elem, r0, pad;
};

struct BParams {
  const BGroup* groups;
  const BItem* items;
  int32_t nitems;
  int32_t* counter;           // queue head
  int32_t m, max_iters, max_outer, mixed;
  double rtol, inner_rtol;
  char* slots;                // per lane group: vectors and scalars (slot_layout)
  BatchStats* st;
};

// ---- shared-memory image of one element (offsets in T) -----------------------
struct ElemLayout {
  int SA, SB, Q1, Q2, T1, T2, Azi, D, w, l0, l1, cx, cy, cz, fa, total;
};

// factors = false: the operator's data only (the FP64 image of the mixed mode)
__host__ __device__ inline ElemLayout elem_layout(int dim, int nmax, bool factors) {
  const int nn = nmax * nmax, nl = (dim == 2) ? nn : nn * nmax, nf = (dim == 2) ? nmax : nn;
  const int nfac = factors ? nn : 0;
  ElemLayout L;
  int o = 0;
  L.SA = o; o += nfac;
  L.SB = o; o += nfac;
  L.Q1 = o; o += nfac;
  L.Q2 = o; o += nfac;
  L.T1 = o; o += nfac;
  L.T2 = o; o += nfac;
  L.Azi = o; o += (dim == 3) ? nfac : 0;
  L.D = o; o += nn;
  L.w = o; o += nmax;
  L.l0 = o; o += nmax;
  L.l1 = o; o += nmax;
  L.cx = o; o += nl;
  L.cy = o; o += nl;
  L.cz = o; o += (dim == 3) ? nl : 0;
  L.fa = o; o += 2 * dim * nf;
  L.total = o;
  return L;
}

// block structure of the quasi-triangular T2 (rows) and T1 (columns)
struct BlockIdx {
  int rs[33], cs[33], colblk[32], nbr, nbc;
};

template <typename T>
__device__ void stage_element(const BGroup& G, const GroupData<T>& D, int64_t e, T* sm,
                              const ElemLayout& L, BlockIdx* bi, bool factors) {
  const int n = G.n, nn = n * n, nl = G.nloc, tid = threadIdx.x, nt = blockDim.x;
  const int nf = (G.dim == 2) ? n : nn;
  const int64_t gf = e * nn, gl = e * nl;
  for (int q = tid; q < nn; q += nt) {
    if (factors) {
      sm[L.SA + q] = D.SA[gf + q];
      sm[L.SB + q] = D.SB[gf + q];
      sm[L.Q1 + q] = D.Q1[gf + q];
      sm[L.Q2 + q] = D.Q2[gf + q];
      sm[L.T1 + q] = D.T1[gf + q];
      sm[L.T2 + q] = D.T2[gf + q];
      if (G.dim == 3) sm[L.Azi + q] = D.Azi[gf + q];
    }
    sm[L.D + q] = (T)G.T->D[q];
  }
  for (int q = tid; q < n; q += nt) {
    sm[L.w + q] = (T)G.T->w[q];
    sm[L.l0 + q] = (T)G.T->l0[q];
    sm[L.l1 + q] = (T)G.T->l1[q];
  }
  for (int q = tid; q < nl; q += nt) {
    sm[L.cx + q] = D.cx[gl + q];
    sm[L.cy + q] = D.cy[gl + q];
    if (G.dim == 3) sm[L.cz + q] = D.cz[gl + q];
  }
  for (int q = tid; q < 2 * G.dim * nf; q += nt) {      // outflow part only (isolated)
    const T a = D.fa[e * 2 * G.dim * nf + q];
    sm[L.fa + q] = a > (T)0 ? a : (T)0;
  }
  if (factors && tid == 0) {
    const uint32_t m2 = G.masks[2 * e + 1], m1 = G.masks[2 * e];
    int nb = 0, r = 0;
    while (r < n) {
      bi->rs[nb++] = r;
      r += (((m2 >> r) & 1u) && r + 1 < n) ? 2 : 1;
    }
    bi->rs[nb] = n;
    bi->nbr = nb;
    nb = 0;
    r = 0;
    while (r < n) {
      bi->cs[nb] = r;
      const int w = (((m1 >> r) & 1u) && r + 1 < n) ? 2 : 1;
      for (int t = 0; t < w; ++t) bi->colblk[r + t] = nb;
      ++nb;
      r += w;
    }
    bi->cs[nb] = n;
    bi->nbc = nb;
  }
}

// ---- lane-group reductions ----------------------------------------------------
template <int NM, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned gmask) {
#pragma unroll
  for (int o = NM / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o);
  return v;
}

// ---- operator, one 2D block: y = h^2 (w (x) w) x + volume + outflow faces (the
// isolated diagonal block of Sec. 3.4.1's Jacobian, as in k_dg_apply_2d):
//   y_ij = hd w_i w_j x_ij + sum_k D_ki cx_kj x_kj + sum_l D_lj cy_il x_il
//          + l0_i F-x_j + l1_i F+x_j + l0_j F-y_i + l1_j F+y_i,  F_f = max(fa_f, 0) u_f.
// x, y: global (vector block of the system); Wm: n*n of shared scratch of the group.
template <typename T, int NM>
__device__ __noinline__ void op_2d(const T* sm, const ElemLayout& L, int n, T hd, const T* __restrict__ x,
                      T* __restrict__ y, T* Wm, int i, unsigned gmask, int lbase) {
  const bool rok = i < n;
  T xr[NM];
#pragma unroll
  for (int j = 0; j < NM; ++j) xr[j] = (rok && j < n) ? x[i + n * j] : (T)0;
#pragma unroll
  for (int j = 0; j < NM; ++j)
    if (rok && j < n) Wm[i + n * j] = xr[j];
  __syncwarp(gmask);
  // traces: y-faces along the own row, x-faces along column i (lane i = column index)
  T uy0 = 0, uy1 = 0, ux0 = 0, ux1 = 0;
  if (rok) {
#pragma unroll
    for (int j = 0; j < NM; ++j)
      if (j < n) {
        uy0 += sm[L.l0 + j] * xr[j];
        uy1 += sm[L.l1 + j] * xr[j];
      }
    for (int k = 0; k < n; ++k) {
      const T v = Wm[k + n * i];
      ux0 += sm[L.l0 + k] * v;
      ux1 += sm[L.l1 + k] * v;
    }
  }
  const T Fx0 = rok ? sm[L.fa + 0 * n + i] * ux0 : (T)0;
  const T Fx1 = rok ? sm[L.fa + 1 * n + i] * ux1 : (T)0;
  const T Fy0 = rok ? sm[L.fa + 2 * n + i] * uy0 : (T)0;
  const T Fy1 = rok ? sm[L.fa + 3 * n + i] * uy1 : (T)0;
  __syncwarp(gmask);
#pragma unroll
  for (int j = 0; j < NM; ++j)
    if (rok && j < n) Wm[i + n * j] = sm[L.cx + i + n * j] * xr[j];
  __syncwarp(gmask);
  const T wi = rok ? hd * sm[L.w + i] : (T)0, l0i = rok ? sm[L.l0 + i] : (T)0,
          l1i = rok ? sm[L.l1 + i] : (T)0;
  T pyr[NM];                                     // cy * x along the own row
#pragma unroll
  for (int l = 0; l < NM; ++l) pyr[l] = (rok && l < n) ? sm[L.cy + i + n * l] * xr[l] : (T)0;
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    if (j < n) {
      const T fx0 = __shfl_sync(gmask, Fx0, lbase + j);
      const T fx1 = __shfl_sync(gmask, Fx1, lbase + j);
      if (rok) {
        T acc = wi * sm[L.w + j] * xr[j];
        for (int k = 0; k < n; ++k) acc += sm[L.D + k * n + i] * Wm[k + n * j];
#pragma unroll
        for (int l = 0; l < NM; ++l)
          if (l < n) acc += sm[L.D + l * n + j] * pyr[l];
        acc += l0i * fx0 + l1i * fx1 + sm[L.l0 + j] * Fy0 + sm[L.l1 + j] * Fy1;
        y[i + n * j] = acc;
      }
    }
  }
  __syncwarp(gmask);
}

// Solve T2_II Y + Y T1_JJ^T = R for one ni x nj diagonal block pair (ni, nj in
// {1, 2}); a = T2_II (a[r + 2 c]), bt = T1_JJ; y in: R, out: Y (column-major, ld ni)
template <typename T>
__device__ __forceinline__ void block_sylvester(int ni, int nj, const T a[4], const T bt[4],
                                                T y[4]) {
  if (ni == 1 && nj == 1) {
    y[0] = y[0] / (a[0] + bt[0]);
  } else if (nj == 1 || ni == 1) {      // (M + s I) y = r with M the 2x2 block
    const T* M = (nj == 1) ? a : bt;
    const T sft = (nj == 1) ? bt[0] : a[0];
    const T m00 = M[0] + sft, m01 = M[2], m10 = M[1], m11 = M[3] + sft;
    const T det = m00 * m11 - m01 * m10;
    const T y0 = (m11 * y[0] - m01 * y[1]) / det;
    const T y1 = (m00 * y[1] - m10 * y[0]) / det;
    y[0] = y0;
    y[1] = y1;
  } else {                               // (I (x) A + B (x) I) vec(Y) = vec(R), 4 x 4, GEPP
    T M[4][5];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int r = p & 1, c = p >> 1;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r2 = q & 1, c2 = q >> 1;
        M[p][q] = (c == c2 ? a[r + 2 * r2] : (T)0) + (r == r2 ? bt[c + 2 * c2] : (T)0);
      }
      M[p][4] = y[p];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int i = k + 1; i < 4; ++i)
        if (fabs((double)M[i][k]) > fabs((double)M[k][k])) {
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            const T t = M[k][q];
            M[k][q] = M[i][q];
            M[i][q] = t;
          }
        }
#pragma unroll
      for (int i = k + 1; i < 4; ++i) {
        const T f = M[i][k] / M[k][k];
#pragma unroll
        for (int q = k; q < 5; ++q) M[i][q] -= f * M[k][q];
      }
    }
#pragma unroll
    for (int k = 3; k >= 0; --k) {
      T acc = M[k][4];
#pragma unroll
      for (int q = k + 1; q < 4; ++q) acc -= M[k][q] * y[q];
      y[k] = acc / M[k][k];
    }
  }
}

// ---- preconditioner, one 2D block (Alg. 2d-apply, two-sided form):
//   C = S_B B S_A^T,  T_2 Y + Y T_1^T = C (quasi-triangular, anti-diagonal wavefront over
//   the 1x1 / 2x2 block grid),  x = Q_2 Y Q_1^T.
// Lane i of the group owns row i; b and x may alias (each lane reads its row first).
template <typename T, int NM>
__device__ __noinline__ void apply_2d(const T* sm, const ElemLayout& L, const BlockIdx& bi, int n,
                         const T* b, T* x, T* Wm, int i, unsigned gmask, int lbase) {
  const bool rok = i < n;
  const T* SA = sm + L.SA;
  const T* SB = sm + L.SB;
  const T* T1 = sm + L.T1;
  const T* T2 = sm + L.T2;
  T row[NM], acc[NM];
#pragma unroll
  for (int k = 0; k < NM; ++k) row[k] = (rok && k < n) ? b[i + n * k] : (T)0;
  __syncwarp(gmask);
  // W = B S_A^T
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    if (j < n) {
      T s = (T)0;
#pragma unroll
      for (int k = 0; k < NM; ++k)
        if (k < n) s += row[k] * SA[j + n * k];
      if (rok) Wm[i + n * j] = s;
    }
  }
  __syncwarp(gmask);
  // C = S_B W, row i in registers
#pragma unroll
  for (int k = 0; k < NM; ++k) row[k] = (rok && k < n) ? SB[i + n * k] : (T)0;
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    T s = (T)0;
    if (j < n) {
#pragma unroll
      for (int k = 0; k < NM; ++k)
        if (k < n) s += row[k] * Wm[k + n * j];
    }
    acc[j] = s;
  }
  __syncwarp(gmask);
  // Sylvester T2 Y + Y T1^T = C
  {
    const int nbr = bi.nbr, nbc = bi.nbc;
    int I = 0;
    if (rok)
      while (bi.rs[I + 1] <= i) ++I;
    const int i0 = rok ? bi.rs[I] : 0, ni = rok ? bi.rs[I + 1] - i0 : 1;
    const int aI = nbr - 1 - I;
    const int partner = (ni == 2) ? lbase + ((i == i0) ? i0 + 1 : i0) : lbase + i;
    const T t2ii = rok ? T2[i + n * i] : (T)1;
    int aJ[NM];
#pragma unroll
    for (int j = 0; j < NM; ++j) aJ[j] = (j < n) ? nbc - 1 - bi.colblk[j] : 0;
    const int steps = nbr + nbc - 1;
    for (int st = 0; st < steps; ++st) {
      const int bJ = st - aI;
      const bool act = rok && bJ >= 0 && bJ < nbc;
      int j0 = 0, nj = 1;
      if (act) {
        const int Js = nbc - 1 - bJ;
        j0 = bi.cs[Js];
        nj = bi.cs[Js + 1] - j0;
      }
      T r0 = (T)0, r1 = (T)0;
#pragma unroll
      for (int j = 0; j < NM; ++j) {
        if (j == j0) r0 = acc[j];
        if (j == j0 + 1) r1 = acc[j];
      }
      const T p0 = __shfl_sync(gmask, r0, partner & 31);
      const T p1 = __shfl_sync(gmask, r1, partner & 31);
      T y0 = (T)0, y1 = (T)0;
      if (act) {
        if (ni == 1 && nj == 1) {
          y0 = r0 / (t2ii + T1[j0 + n * j0]);
        } else {
          T ab[4] = {T2[i0 + n * i0], (T)0, (T)0, (T)0};
          T bb[4] = {T1[j0 + n * j0], (T)0, (T)0, (T)0};
          T rhs[4] = {(T)0, (T)0, (T)0, (T)0};
          const int rr = i - i0;
          if (ni == 2) {
            ab[1] = T2[(i0 + 1) + n * i0];
            ab[2] = T2[i0 + n * (i0 + 1)];
            ab[3] = T2[(i0 + 1) + n * (i0 + 1)];
            rhs[rr] = r0;
            rhs[1 - rr] = p0;
            if (nj == 2) {
              rhs[2 + rr] = r1;
              rhs[2 + 1 - rr] = p1;
            }
          } else {
            rhs[0] = r0;
            if (nj == 2) rhs[1] = r1;
          }
          if (nj == 2) {
            bb[1] = T1[(j0 + 1) + n * j0];
            bb[2] = T1[j0 + n * (j0 + 1)];
            bb[3] = T1[(j0 + 1) + n * (j0 + 1)];
          }
          block_sylvester<T>(ni, nj, ab, bb, rhs);
          y0 = rhs[rr];
          if (nj == 2) y1 = rhs[rr + ni];
        }
      }
#pragma unroll
      for (int j = 0; j < NM; ++j) {
        if (act && j == j0) acc[j] = y0;
        if (act && nj == 2 && j == j0 + 1) acc[j] = y1;
      }
      if (st + 1 < steps) {
#pragma unroll
        for (int j = 0; j < NM; ++j) {
          if (j < n) {
            const int a = st - aJ[j];
            const bool valid = a >= 0 && a < nbr;
            const bool unsolved = rok && (aI + aJ[j] > st);
            T v = (T)0;
            if (valid) {
              const int ks = bi.rs[nbr - 1 - a];
              const int nks = bi.rs[nbr - a] - ks;
              const T yk0 = __shfl_sync(gmask, acc[j], (lbase + ks) & 31);
              const T yk1 = __shfl_sync(gmask, acc[j], (lbase + ks + (nks - 1)) & 31);
              if (unsolved) {
                v += T2[i + n * ks] * yk0;
                if (nks == 2) v += T2[i + n * (ks + 1)] * yk1;
              }
            }
            if (act && unsolved) {
              v += y0 * T1[j + n * j0];
              if (nj == 2) v += y1 * T1[j + n * (j0 + 1)];
            }
            acc[j] -= v;
          }
        }
      }
    }
  }
  __syncwarp(gmask);
  // W = Y Q1^T
  const T* Q1 = sm + L.Q1;
  const T* Q2 = sm + L.Q2;
#pragma unroll
  for (int k = 0; k < NM; ++k) row[k] = (rok && k < n) ? acc[k] : (T)0;
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    if (j < n) {
      T s = (T)0;
#pragma unroll
      for (int k = 0; k < NM; ++k)
        if (k < n) s += row[k] * Q1[j + n * k];
      if (rok) Wm[i + n * j] = s;
    }
  }
  __syncwarp(gmask);
  // x = Q2 W
#pragma unroll
  for (int k = 0; k < NM; ++k) row[k] = (rok && k < n) ? Q2[i + n * k] : (T)0;
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    if (j < n) {
      T s = (T)0;
#pragma unroll
      for (int k = 0; k < NM; ++k)
        if (k < n) s += row[k] * Wm[k + n * j];
      if (rok) x[i + n * j] = s;
    }
  }
  __syncwarp(gmask);
}

// ---- operator, one 3D block (as in k_dg_apply_3d, isolated): lanes stride over the
// n^3 outputs, x read through L1; Fs: 6 n^2 scratch (global slot) for the face fluxes
template <typename T, int NM>
__device__ __noinline__ void op_3d(const T* sm, const ElemLayout& L, int n, T hd, const T* __restrict__ x,
                      T* __restrict__ y, T* Fs, int gl, unsigned gmask) {
  const int nn = n * n, n3 = nn * n;
  const T* l0 = sm + L.l0;
  const T* l1 = sm + L.l1;
  const T* fa = sm + L.fa;
  for (int t = gl; t < nn; t += NM) {
    const int t0 = t % n, t1 = t / n;
    T a0 = 0, a1 = 0, b0 = 0, b1 = 0, c0 = 0, c1 = 0;
    for (int s = 0; s < n; ++s) {
      const T vx = x[s + n * t0 + nn * t1];
      const T vy = x[t0 + n * s + nn * t1];
      const T vz = x[t0 + n * t1 + nn * s];
      a0 += l0[s] * vx; a1 += l1[s] * vx;
      b0 += l0[s] * vy; b1 += l1[s] * vy;
      c0 += l0[s] * vz; c1 += l1[s] * vz;
    }
    Fs[0 * nn + t] = fa[0 * nn + t] * a0;
    Fs[1 * nn + t] = fa[1 * nn + t] * a1;
    Fs[2 * nn + t] = fa[2 * nn + t] * b0;
    Fs[3 * nn + t] = fa[3 * nn + t] * b1;
    Fs[4 * nn + t] = fa[4 * nn + t] * c0;
    Fs[5 * nn + t] = fa[5 * nn + t] * c1;
  }
  __syncwarp(gmask);
  const T* D = sm + L.D;
  const T* w = sm + L.w;
  const T* cx = sm + L.cx;
  const T* cy = sm + L.cy;
  const T* cz = sm + L.cz;
  for (int q = gl; q < n3; q += NM) {
    const int i = q % n, j = (q / n) % n, k = q / nn;
    T acc = hd * w[i] * w[j] * w[k] * x[q];
    const int rx = n * j + nn * k, ry = i + nn * k, rz = i + n * j;
    for (int a = 0; a < n; ++a) acc += D[a * n + i] * cx[a + rx] * x[a + rx];
    for (int b = 0; b < n; ++b) acc += D[b * n + j] * cy[ry + n * b] * x[ry + n * b];
    for (int c = 0; c < n; ++c) acc += D[c * n + k] * cz[rz + nn * c] * x[rz + nn * c];
    const int qx = j + n * k, qy = i + n * k, qz = i + n * j;
    acc += l0[i] * Fs[0 * nn + qx] + l1[i] * Fs[1 * nn + qx];
    acc += l0[j] * Fs[2 * nn + qy] + l1[j] * Fs[3 * nn + qy];
    acc += l0[k] * Fs[4 * nn + qz] + l1[k] * Fs[5 * nn + qz];
    y[q] = acc;
  }
  __syncwarp(gmask);
}

// ---- preconditioner, one 3D block (Alg. 3d-apply, nested): x~ = (A1^-1 (x) I) b along
// z, then the 2D apply of D1^-1 on every z slice, in place
template <typename T, int NM>
__device__ __noinline__ void apply_3d(const T* sm, const ElemLayout& L, const BlockIdx& bi, int n,
                         const T* b, T* x, T* Wm, int gl, unsigned gmask, int lbase) {
  const int nn = n * n;
  const T* az = sm + L.Azi;
  for (int q = gl; q < nn; q += NM) {
    T line[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) line[k] = (k < n) ? b[q + nn * k] : (T)0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k < n) {
        T s = (T)0;
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2)
          if (k2 < n) s += az[k + n * k2] * line[k2];
        x[q + nn * k] = s;
      }
    }
  }
  __syncwarp(gmask);
  for (int k = 0; k < n; ++k)
    apply_2d<T, NM>(sm, L, bi, n, x + nn * k, x + nn * k, Wm, gl, gmask, lbase);
}

// per-system view handed to the Krylov routine
template <typename T, int NM>
struct SysCtx {
  const T* sm;              // element image (this precision)
  ElemLayout L;
  const BlockIdx* bi;
  int dim, n, nloc;
  T hd;
  T* Wm;                    // n^2 shared scratch of the lane group
  T* Fs;                    // 6 n^2 global scratch (3D face fluxes)
  int gl, lbase;
  unsigned gmask;

  // the 32-lane launch serves 2D groups only (3D n <= 16)
  __device__ void op(const T* x, T* y) const {
    if (NM == 32 || dim == 2) op_2d<T, NM>(sm, L, n, hd, x, y, Wm, gl, gmask, lbase);
    else op_3d<T, NM>(sm, L, n, hd, x, y, Fs, gl, gmask);
  }
  __device__ void prec(const T* b, T* x) const {
    if (NM == 32 || dim == 2) apply_2d<T, NM>(sm, L, *bi, n, b, x, Wm, gl, gmask, lbase);
    else apply_3d<T, NM>(sm, L, *bi, n, b, x, Wm, gl, gmask, lbase);
  }
  __device__ double dot(const T* a, const T* b) const {
    T s = (T)0;
    for (int q = gl; q < nloc; q += NM) s += a[q] * b[q];
    return (double)group_sum<NM>(s, gmask);
  }
};

// ---- right-preconditioned restarted GMRES(m) for one system, from sol = 0:
// S sol = rhs to ||rhs - S sol|| <= rtol ||rhs|| or max_it Arnoldi steps.  Classical
// Gram-Schmidt with one reorthogonalisation pass; Hessenberg columns reduced by
// Givens rotations as they are formed (the group's first lane); the update
// sol += P^-1 (V y) once per cycle, then the true residual.  V: (m+1) nloc, Z, W: nloc
// (all of type T, global slot); Hs: (m+1) m + 4 m + 3 doubles.  Returns the number
// of Arnoldi steps; *rel = final true relative residual.
template <typename T, int NM>
__device__ __noinline__ int gmres_sys(const SysCtx<T, NM>& c, const T* rhs, T* sol, double rtol, int m,
                         int max_it, T* V, T* Z, T* W, double* Hs, double* rel) {
  const int nloc = c.nloc, gl = c.gl;
  const unsigned gmask = c.gmask;
  const int lead = c.lbase;
  double* H = Hs;                       // (m+1) x m, column j at H + (m+1) j
  double* cs = H + (m + 1) * m;
  double* sn = cs + m;
  double* g = sn + m;                   // m + 1
  double* hv = g + m + 1;               // m + 2: projections of a pass, then y
  for (int q = gl; q < nloc; q += NM) sol[q] = (T)0;
  __syncwarp(gmask);
  const double beta0 = sqrt(c.dot(rhs, rhs));
  if (!(beta0 > 0.0)) {
    *rel = 0.0;
    return 0;
  }
  const T* r = rhs;                     // later cycles: r = rhs - S sol in W
  double beta = beta0;
  int it = 0;
  while (true) {
    {
      const T inv = (T)(1.0 / beta);
      for (int q = gl; q < nloc; q += NM) V[q] = r[q] * inv;
    }
    if (gl == 0) {
      g[0] = beta;
      for (int k = 1; k <= m; ++k) g[k] = 0.0;
    }
    __syncwarp(gmask);
    int jn = 0;
    for (int j = 0; j < m && it < max_it; ++j) {
      T* Vj = V + (size_t)j * nloc;
      T* Vn = Vj + nloc;
      c.prec(Vj, Z);
      c.op(Z, W);
      // CGS2: each pass takes all j + 1 projections in one sweep over W and the basis,
      // then subtracts them in a second sweep (which also sums ||W||^2 after pass 2)
      double hn2 = 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        T acc[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) acc[k] = (T)0;
        for (int q = gl; q < nloc; q += NM) {
          const T w = W[q];
#pragma unroll
          for (int k = 0; k < 32; ++k)
            if (k <= j) acc[k] += V[(size_t)k * nloc + q] * w;
        }
#pragma unroll
        for (int k = 0; k < 32; ++k)
          if (k <= j) acc[k] = group_sum<NM>(acc[k], gmask);
        T n2 = (T)0;
        for (int q = gl; q < nloc; q += NM) {
          T s = W[q];
#pragma unroll
          for (int k = 0; k < 32; ++k)
            if (k <= j) s -= acc[k] * V[(size_t)k * nloc + q];
          W[q] = s;
          n2 += s * s;
        }
        if (gl == 0) {
          double* Hj = H + (m + 1) * j;
#pragma unroll
          for (int k = 0; k < 32; ++k)
            if (k <= j) Hj[k] = (pass == 0) ? (double)acc[k] : Hj[k] + (double)acc[k];
        }
        if (pass == 1) hn2 = (double)group_sum<NM>(n2, gmask);
        __syncwarp(gmask);
      }
      const double hn = sqrt(hn2);
      {
        const T inv = (hn > 0.0) ? (T)(1.0 / hn) : (T)0;
        for (int q = gl; q < nloc; q += NM) Vn[q] = W[q] * inv;
      }
      double res = 0.0;
      if (gl == 0) {
        double* Hj = H + (m + 1) * j;
        Hj[j + 1] = hn;
        for (int k = 0; k < j; ++k) {
          const double t = cs[k] * Hj[k] + sn[k] * Hj[k + 1];
          Hj[k + 1] = -sn[k] * Hj[k] + cs[k] * Hj[k + 1];
          Hj[k] = t;
        }
        const double a = Hj[j], bb = Hj[j + 1];
        const double rr = sqrt(a * a + bb * bb);
        const double cc = (rr > 0.0) ? a / rr : 1.0, ss = (rr > 0.0) ? bb / rr : 0.0;
        cs[j] = cc;
        sn[j] = ss;
        Hj[j] = rr;
        Hj[j + 1] = 0.0;
        g[j + 1] = -ss * g[j];
        g[j] = cc * g[j];
        res = fabs(g[j + 1]);
      }
      res = __shfl_sync(gmask, res, lead);
      __syncwarp(gmask);
      ++it;
      jn = j + 1;
      if (res <= rtol * beta0 || !(hn > 0.0)) break;
    }
    // y = R^-1 g (back substitution), U = V y into W, sol += P^-1 U
    if (gl == 0) {
      for (int k = jn - 1; k >= 0; --k) {
        double s = g[k];
        for (int l = k + 1; l < jn; ++l) s -= H[(m + 1) * l + k] * hv[l];
        const double d = H[(m + 1) * k + k];
        hv[k] = (d != 0.0) ? s / d : 0.0;
      }
    }
    __syncwarp(gmask);
    for (int q = gl; q < nloc; q += NM) {
      T s = (T)0;
      for (int k = 0; k < jn; ++k) s += V[(size_t)k * nloc + q] * (T)hv[k];
      W[q] = s;
    }
    __syncwarp(gmask);
    c.prec(W, Z);
    for (int q = gl; q < nloc; q += NM) sol[q] += Z[q];
    __syncwarp(gmask);
    c.op(sol, W);                                        // true residual
    for (int q = gl; q < nloc; q += NM) W[q] = rhs[q] - W[q];
    __syncwarp(gmask);
    beta = sqrt(c.dot(W, W));
    r = W;
    if (beta <= rtol * beta0 || it >= max_it || jn == 0) break;
  }
  *rel = beta / beta0;
  return it;
}

// ---- per lane-group slot of global memory (byte offsets, 256-aligned) ------------
struct SlotLayout {
  size_t Hs, Fs, V, Z, W, rf, df, r64, total;
};

__host__ __device__ inline size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

__host__ __device__ inline SlotLayout slot_layout(int m, int nloc, int nmax, bool mixed) {
  const size_t ts = mixed ? 4 : 8;
  SlotLayout S;
  size_t o = 0;
  S.Hs = o; o += al256((size_t)((m + 1) * m + 4 * m + 3) * 8);
  S.Fs = o; o += al256((size_t)6 * nmax * nmax * 8);
  S.V = o; o += al256((size_t)(m + 1) * nloc * ts);
  S.Z = o; o += al256((size_t)nloc * ts);
  S.W = o; o += al256((size_t)nloc * ts);
  S.rf = o; o += mixed ? al256((size_t)nloc * 4) : 0;
  S.df = o; o += mixed ? al256((size_t)nloc * 4) : 0;
  S.r64 = o; o += mixed ? al256((size_t)nloc * 8) : 0;
  S.total = o;
  return S;
}

template <typename T> struct Pick;
template <> struct Pick<double> {
  static __device__ const GroupData<double>& of(const BGroup& G) { return G.d64; }
};
template <> struct Pick<float> {
  static __device__ const GroupData<float>& of(const BGroup& G) { return G.d32; }
};

__device__ inline void atomic_max_nonneg(double* a, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

struct ClassArgs {
  int max_nloc, max_n;
};

// MINB: register budget, at least MINB resident CTAs of 256 threads per SM
template <int NM, bool MIXED, int MINB>
__global__ void __launch_bounds__(256, MINB) k_bgmres(BParams P, ClassArgs C) {
  using TI = typename std::conditional<MIXED, float, double>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ BlockIdx bi;
  __shared__ int s_item;
  constexpr int EPW = 32 / NM;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  const int gslot = lane / NM, gl = lane % NM, lbase = gslot * NM;
  const unsigned gmask = (NM == 32) ? 0xffffffffu : (((1u << NM) - 1u) << lbase);
  const int gidx = warp * EPW + gslot, ngc = nw * EPW;
  double* scratch = reinterpret_cast<double*>(smraw) + (size_t)gidx * NM * NM;
  unsigned char* img = smraw + (size_t)ngc * NM * NM * 8;
  const SlotLayout SL = slot_layout(P.m, C.max_nloc, C.max_n, MIXED);
  char* my = P.slots + ((size_t)blockIdx.x * ngc + gidx) * SL.total;
  double* Hs = reinterpret_cast<double*>(my + SL.Hs);
  while (true) {
    __syncthreads();                      // the previous element is done with smem
    if (tid == 0) s_item = atomicAdd(P.counter, 1);
    __syncthreads();
    const int itm = s_item;
    if (itm >= P.nitems) break;
    const BItem I = P.items[itm];
    const BGroup& G = P.groups[I.group];
    const ElemLayout Li = elem_layout(G.dim, G.n, true);
    TI* smi = reinterpret_cast<TI*>(img);
    stage_element<TI>(G, Pick<TI>::of(G), I.elem, smi, Li, &bi, true);
    const ElemLayout L64 = elem_layout(G.dim, G.n, false);
    double* sm64 = reinterpret_cast<double*>(img + al256((size_t)Li.total * sizeof(TI)));
    if (MIXED) stage_element<double>(G, G.d64, I.elem, sm64, L64, &bi, false);
    __syncthreads();
    SysCtx<TI, NM> ci;
    ci.sm = smi; ci.L = Li; ci.bi = &bi; ci.dim = G.dim; ci.n = G.n; ci.nloc = G.nloc;
    ci.hd = (TI)G.hd; ci.Wm = reinterpret_cast<TI*>(scratch);
    ci.Fs = reinterpret_cast<TI*>(my + SL.Fs); ci.gl = gl; ci.lbase = lbase; ci.gmask = gmask;
    for (int r = I.r0 + gidx; r < G.R && r < I.r0 + ngc; r += ngc) {
      const int64_t off = ((int64_t)I.elem * G.R + r) * G.nloc;
      const double* b64 = G.b + off;
      double* x64 = G.x + off;
      double rel = 0.0;
      int its = 0, outer = 0;
      if constexpr (!MIXED) {
        its = gmres_sys<TI, NM>(ci, b64, x64, P.rtol, P.m, P.max_iters,
                                reinterpret_cast<TI*>(my + SL.V), reinterpret_cast<TI*>(my + SL.Z),
                                reinterpret_cast<TI*>(my + SL.W), Hs, &rel);
        outer = 1;
      } else {
        SysCtx<double, NM> c64;
        c64.sm = sm64; c64.L = L64; c64.bi = &bi; c64.dim = G.dim; c64.n = G.n;
        c64.nloc = G.nloc; c64.hd = G.hd; c64.Wm = scratch;
        c64.Fs = reinterpret_cast<double*>(my + SL.Fs); c64.gl = gl; c64.lbase = lbase;
        c64.gmask = gmask;
        float* rf = reinterpret_cast<float*>(my + SL.rf);
        float* df = reinterpret_cast<float*>(my + SL.df);
        double* r64 = reinterpret_cast<double*>(my + SL.r64);
        const int nl = G.nloc;
        for (int q = gl; q < nl; q += NM) {
          x64[q] = 0.0;
          r64[q] = b64[q];
        }
        __syncwarp(gmask);
        const double beta0 = sqrt(c64.dot(b64, b64));
        double beta = beta0;
        while (beta > P.rtol * beta0 && outer < P.max_outer && its < P.max_iters) {
          const float inv = (float)(1.0 / beta);
          for (int q = gl; q < nl; q += NM) rf[q] = (float)r64[q] * inv;
          __syncwarp(gmask);
          double rin = 0.0;
          its += gmres_sys<float, NM>(ci, rf, df, P.inner_rtol, P.m, P.max_iters - its,
                                      reinterpret_cast<float*>(my + SL.V),
                                      reinterpret_cast<float*>(my + SL.Z),
                                      reinterpret_cast<float*>(my + SL.W), Hs, &rin);
          for (int q = gl; q < nl; q += NM) x64[q] += beta * (double)df[q];
          __syncwarp(gmask);
          c64.op(x64, r64);
          for (int q = gl; q < nl; q += NM) r64[q] = b64[q] - r64[q];
          __syncwarp(gmask);
          beta = sqrt(c64.dot(r64, r64));
          ++outer;
        }
        rel = (beta0 > 0.0) ? beta / beta0 : 0.0;
      }
      if (gl == 0) {
        const int64_t sidx = (int64_t)I.elem * G.R + r;
        if (G.iters) G.iters[sidx] = its;
        if (G.relres) G.relres[sidx] = rel;
        atomicAdd(&P.st->total_iters, (unsigned long long)its);
        atomicMax(&P.st->max_iters, its);
        atomicMax(&P.st->outer_max, outer);
        if (!(rel <= P.rtol)) atomicAdd(&P.st->unconverged, 1);
        atomic_max_nonneg(&P.st->max_relres, rel);
      }
      __syncwarp(gmask);
    }
  }
}

// kernels of one lane-group width (defined in k_bgmres_w8.cu, _w16.cu, _w32.cu)
const void* kernel_w8(bool mixed, int minb);
const void* kernel_w16(bool mixed, int minb);
const void* kernel_w32(bool mixed, int minb);

}  // namespace bg
}  // namespace tpp
