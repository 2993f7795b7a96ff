// Application of the Kronecker preconditioner, x = P^-1 b (Alg. 2d-apply).
//
// With B the n x n matrix of b (B[i, j] = b[i + n j], rows = x index) and
// (A (x) B) vec(X) = vec(B X A^T):
//   C = S_B B S_A^T                 (S_A = Q_1^T L_A^-1, S_B = Q_2^T L_B^-1)
//   T_2 Y + Y T_1^T = C             (quasi-triangular Sylvester, Eq. quad-triang)
//   X = Q_2 Y Q_1^T.
// One CTA per element, factors staged through shared memory in the order the
// stages consume them.  The Sylvester system is solved by a wavefront over
// the 1x1 / 2x2 diagonal blocks of T_2 (rows) and T_1 (columns): block (I, J)
// depends only on blocks below it in its column and right of it in its row.
#include "tpp_internal.cuh"

namespace tpp {

namespace {


// Solve T2_II Y + Y T1_JJ^T = R for one ni x nj diagonal block pair
// (ni, nj in {1, 2}); a = T2_II (a[r + 2 c]), bt = T1_JJ, y in: R, out: Y
// (column-major, ld ni).  Written out per shape so everything stays in
// registers; the 2x2-by-2x2 case is a 4 x 4 system solved by Gaussian
// elimination with partial pivoting.
template <typename T>
__device__ __forceinline__ void small_sylvester(int ni, int nj, const T a[4], const T bt[4],
                                                T y[4]) {
  if (ni == 1 && nj == 1) {
    y[0] = y[0] / (a[0] + bt[0]);
  } else if (nj == 1) {            // (A + b I) y = r, A 2x2
    const T m00 = a[0] + bt[0], m01 = a[2], m10 = a[1], m11 = a[3] + bt[0];
    const T det = m00 * m11 - m01 * m10;
    const T y0 = (m11 * y[0] - m01 * y[1]) / det;
    const T y1 = (m00 * y[1] - m10 * y[0]) / det;
    y[0] = y0;
    y[1] = y1;
  } else if (ni == 1) {            // y (B^T + a I) = r: (B + a I) y^T = r^T
    const T m00 = bt[0] + a[0], m01 = bt[2], m10 = bt[1], m11 = bt[3] + a[0];
    const T det = m00 * m11 - m01 * m10;
    const T y0 = (m11 * y[0] - m01 * y[1]) / det;
    const T y1 = (m00 * y[1] - m10 * y[0]) / det;
    y[0] = y0;
    y[1] = y1;
  } else {                          // (I (x) A + B (x) I) vec(Y) = vec(R), 4 x 4
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
      for (int i = k + 1; i < 4; ++i) {
        if (fabs((double)M[i][k]) > fabs((double)M[k][k])) {
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            const T t = M[k][q];
            M[k][q] = M[i][q];
            M[i][q] = t;
          }
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

}  // namespace

// ---------------------------------------------------------------------------
// One element per group of NM lanes (NM = 8, 16 or 32 >= n; 32 / NM elements
// per warp), lane i owning row i.  Products A B^T / A B keep the row of the
// left operand in registers and read the other operand from shared memory as
// a broadcast; the Sylvester system is solved right-looking over the
// anti-diagonals of the 1x1 / 2x2 block grid: at step s each row block solves
// its block on anti-diagonal s, then every lane updates the unsolved entries
// of its row with the contributions of the blocks solved at step s in their
// columns (T2[i, k] Y[k, j]) and in its own row (Y[i, l] T1[j, l]).  Only
// warp-level synchronisation is needed.
template <typename T, int NM, typename VT>
__global__ void __launch_bounds__(128)
k_apply_2d_w(int n, int64_t E, const T* __restrict__ SA, const T* __restrict__ SB,
             const T* __restrict__ Q1, const T* __restrict__ Q2, const T* __restrict__ T1,
             const T* __restrict__ T2, const uint32_t* __restrict__ masks,
             const VT* b, VT* x, const int32_t* skip, int fdiv) {
  if (skip && *skip) return;
  constexpr int EPW = 32 / NM;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slot = lane / NM, i = lane % NM;
  const int wpb = blockDim.x >> 5;
  const int eslot = warp * EPW + slot;
  const int64_t e = ((int64_t)blockIdx.x * wpb + warp) * EPW + slot;
  const bool eok = e < E;
  const bool rok = eok && i < n;
  const unsigned gmask = (NM == 32) ? 0xffffffffu : (((1u << NM) - 1u) << (slot * NM));
  const int nn = n * n;
  T* Fa = reinterpret_cast<T*>(smraw) + (size_t)eslot * 3 * NM * NM;   // SA, then T2, then Q1
  T* Fb = Fa + NM * NM;                                                  // T1
  T* Wm = Fb + NM * NM;                                                  // work / Y
  int* isx = reinterpret_cast<int*>(reinterpret_cast<T*>(smraw) + (size_t)wpb * EPW * 3 * NM * NM) +
             eslot * (3 * NM + 4);
  int* rs = isx;                  // row block starts (T2), NM + 1
  int* cs = rs + NM + 1;          // column block starts (T1), NM + 1
  int* colblk = cs + NM + 1;      // block of each column, NM
  int* nbs = colblk + NM;         // nbr, nbc
  // vector block e; its factors are those of block e / fdiv (fdiv = 1 in 2D,
  // n in 3D where the blocks are the z slices of an element, in place)
  const int64_t g = eok ? e * nn : 0;
  const int64_t ef = eok ? e / fdiv : 0;
  const int64_t gf = ef * nn;

  // ---- B S_A^T: lane i holds row i of B
  T row[NM], acc[NM];
#pragma unroll
  for (int k = 0; k < NM; ++k) row[k] = (rok && k < n) ? (T)b[g + i + n * k] : (T)0;
  if (eok)
    for (int q = i; q < nn; q += NM) {
      Fa[q] = SA[gf + q];
      Fb[q] = T1[gf + q];
    }
  if (i == 0 && eok) {
    const uint32_t m2 = masks[2 * ef + 1], m1 = masks[2 * ef];
    int nb = 0, r = 0;
    while (r < n) {
      rs[nb++] = r;
      r += (((m2 >> r) & 1u) && r + 1 < n) ? 2 : 1;
    }
    rs[nb] = n;
    nbs[0] = nb;
    nb = 0;
    r = 0;
    while (r < n) {
      cs[nb] = r;
      const int w = (((m1 >> r) & 1u) && r + 1 < n) ? 2 : 1;
      for (int t = 0; t < w; ++t) colblk[r + t] = nb;
      ++nb;
      r += w;
    }
    cs[nb] = n;
    nbs[1] = nb;
  }
  __syncwarp(gmask);
  for (int j = 0; j < n; ++j) {
    T sacc = (T)0;
#pragma unroll
    for (int k = 0; k < NM; ++k)
      if (k < n) sacc += row[k] * Fa[j + n * k];
    if (rok) Wm[i + n * j] = sacc;
  }
  __syncwarp(gmask);
  // ---- C = S_B W: lane i holds row i of S_B; row i of C stays in registers (acc)
#pragma unroll
  for (int k = 0; k < NM; ++k) row[k] = (rok && k < n) ? SB[gf + i + n * k] : (T)0;
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    T sacc = (T)0;
    if (j < n) {
#pragma unroll
      for (int k = 0; k < NM; ++k)
        if (k < n) sacc += row[k] * Wm[k + n * j];
    }
    acc[j] = sacc;
  }
  if (eok)
    for (int q = i; q < nn; q += NM) Fa[q] = T2[gf + q];   // SA no longer needed
  __syncwarp(gmask);

  // ---- Sylvester T2 Y + Y T1^T = C, right-looking wavefront, rows in registers
  {
    const int nbr = eok ? nbs[0] : 1, nbc = eok ? nbs[1] : 1;
    int I = 0;
    if (rok)
      while (rs[I + 1] <= i) ++I;
    const int i0 = rok ? rs[I] : 0, ni = rok ? rs[I + 1] - i0 : 1;
    const int aI = nbr - 1 - I;
    // other row of a 2-row block (own lane otherwise, so every shuffle stays in the group)
    const int partner = (ni == 2) ? slot * NM + ((i == i0) ? i0 + 1 : i0) : lane;
    const T t2ii = rok ? Fa[i + n * i] : (T)1;
    int aJ[NM];                                      // anti-diagonal offset of each column
#pragma unroll
    for (int j = 0; j < NM; ++j) aJ[j] = (eok && j < n) ? nbc - 1 - colblk[j] : 0;
    const int steps = nbr + nbc - 1;
    for (int st = 0; st < steps; ++st) {
      // (A) this row block's block on anti-diagonal st
      const int bJ = st - aI;
      const bool act = rok && bJ >= 0 && bJ < nbc;
      int j0 = 0, nj = 1;
      if (act) {
        const int Js = nbc - 1 - bJ;
        j0 = cs[Js];
        nj = cs[Js + 1] - j0;
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
          y0 = r0 / (t2ii + Fb[j0 + n * j0]);
        } else {
          T ab[4] = {Fa[i0 + n * i0], (T)0, (T)0, (T)0}, bb[4] = {Fb[j0 + n * j0], (T)0, (T)0, (T)0};
          T rhs[4] = {(T)0, (T)0, (T)0, (T)0};
          const int rr = i - i0;
          // rhs column-major (ni x nj): own row from r0/r1, the other row from the partner
          if (ni == 2) {
            ab[1] = Fa[(i0 + 1) + n * i0];
            ab[2] = Fa[i0 + n * (i0 + 1)];
            ab[3] = Fa[(i0 + 1) + n * (i0 + 1)];
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
            bb[1] = Fb[(j0 + 1) + n * j0];
            bb[2] = Fb[j0 + n * (j0 + 1)];
            bb[3] = Fb[(j0 + 1) + n * (j0 + 1)];
          }
          small_sylvester<T>(ni, nj, ab, bb, rhs);
          y0 = rhs[rr];
          if (nj == 2) y1 = rhs[rr + ni];
        }
      }
#pragma unroll
      for (int j = 0; j < NM; ++j) {
        if (act && j == j0) acc[j] = y0;
        if (act && nj == 2 && j == j0 + 1) acc[j] = y1;
      }
      // (B) contributions of the blocks solved at step st to the unsolved entries of row i
      if (st + 1 < steps) {
#pragma unroll
        for (int j = 0; j < NM; ++j) {
          if (j < n) {
            const int a = st - aJ[j];                     // row block solved now in column j
            const bool valid = eok && a >= 0 && a < nbr;   // uniform over the element's lanes
            const bool unsolved = rok && (aI + aJ[j] > st);
            T v = (T)0;
            if (valid) {
              const int ks = rs[nbr - 1 - a];
              const int nks = rs[nbr - a] - ks;
              const T yk0 = __shfl_sync(gmask, acc[j], (slot * NM + ks) & 31);
              const T yk1 = __shfl_sync(gmask, acc[j], (slot * NM + ks + (nks - 1)) & 31);
              if (unsolved) {
                v += Fa[i + n * ks] * yk0;
                if (nks == 2) v += Fa[i + n * (ks + 1)] * yk1;
              }
            }
            if (act && unsolved) {
              v += y0 * Fb[j + n * j0];
              if (nj == 2) v += y1 * Fb[j + n * (j0 + 1)];
            }
            acc[j] -= v;
          }
        }
      }
    }
  }
  __syncwarp(gmask);
  if (eok)
    for (int q = i; q < nn; q += NM) Fa[q] = Q1[gf + q];
  __syncwarp(gmask);
  // ---- W = Y Q1^T: lane i holds row i of Y (acc)
#pragma unroll
  for (int k = 0; k < NM; ++k) row[k] = (rok && k < n) ? acc[k] : (T)0;
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    T sacc = (T)0;
    if (j < n) {
#pragma unroll
      for (int k = 0; k < NM; ++k)
        if (k < n) sacc += row[k] * Fa[j + n * k];
    }
    acc[j] = sacc;
  }
#pragma unroll
  for (int j = 0; j < NM; ++j)
    if (rok && j < n) Wm[i + n * j] = acc[j];
  __syncwarp(gmask);
  // ---- x = Q2 W: lane i holds row i of Q2
#pragma unroll
  for (int k = 0; k < NM; ++k) row[k] = (rok && k < n) ? Q2[gf + i + n * k] : (T)0;
  for (int j = 0; j < n; ++j) {
    T sacc = (T)0;
#pragma unroll
    for (int k = 0; k < NM; ++k)
      if (k < n) sacc += row[k] * Wm[k + n * j];
    if (rok) x[g + i + n * j] = (VT)sacc;
  }
}

// ---------------------------------------------------------------------------
// One-sided form (default).  X solves C2 X + X C1^T = L_B^-1 B L_A^-T; with
// C1 = Q1 T1 Q1^T and Z = X Q1:
//   R = L_B^-1 (B S_A^T)                      (S_A = Q1^T L_A^-1)
//   C2 Z + Z T1^T = R, column blocks of T1 from the last:
//     z_j = Gs_j r^_j + Gp_j r^_p,  r^_l = r_l - sum_{l' > l, outside the block} T1[l, l'] z_l'
//   x = Z Q1^T.
// Layout as in the two-sided kernel: NM lanes per element block, lane i owns
// row i (of B, R, Z, X).  Each column step broadcasts the column's right-hand
// side through shared memory, takes one (two for a 2x2 block) dense n x n
// matvec with the stored inverse (rows read straight from global memory,
// coalesced over the lanes), and updates the remaining columns of its own row
// in registers.  Every FP64 instruction does useful work for all rows; there is
// no per-step division and no cross-row dependency inside a column.
template <typename T, int NM, typename VT>
__global__ void __launch_bounds__(128)
k_apply_2d_g(int n, int64_t E, const T* __restrict__ SA, const T* __restrict__ LBi,
             const T* __restrict__ Q1, const T* __restrict__ T1, const T* __restrict__ G,
             const uint32_t* __restrict__ masks, const VT* b, VT* x,
             const int32_t* skip, int fdiv) {
  if (skip && *skip) return;
  constexpr int EPW = 32 / NM;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slot = lane / NM, i = lane % NM;
  const int wpb = blockDim.x >> 5;
  const int eslot = warp * EPW + slot;
  const int64_t e = ((int64_t)blockIdx.x * wpb + warp) * EPW + slot;
  const bool eok = e < E;
  const bool rok = eok && i < n;
  const unsigned gmask = (NM == 32) ? 0xffffffffu : (((1u << NM) - 1u) << (slot * NM));
  const int nn = n * n;
  T* Fa = reinterpret_cast<T*>(smraw) + (size_t)eslot * 2 * NM * NM;   // S_A, then T1u, then Q1
  T* Wm = Fa + NM * NM;                                                  // work, rhs broadcast
  // vector block e; its factors are those of block e / fdiv (fdiv = 1 in 2D,
  // n in 3D where the blocks are the z slices of an element, in place)
  const int64_t g = eok ? e * nn : 0;
  const int64_t ef = eok ? e / fdiv : 0;
  const int64_t gf = ef * nn;
  const T* Ge = G + (size_t)ef * 2 * n * nn;

  // ---- W = B S_A^T: lane i holds row i of B
  T row[NM], acc[NM];
#pragma unroll
  for (int k = 0; k < NM; ++k) row[k] = (rok && k < n) ? (T)b[g + i + n * k] : (T)0;
  if (eok)
    for (int q = i; q < nn; q += NM) Fa[q] = SA[gf + q];
  __syncwarp(gmask);
  for (int j = 0; j < n; ++j) {
    T sacc = (T)0;
#pragma unroll
    for (int k = 0; k < NM; ++k)
      if (k < n) sacc += row[k] * Fa[j + n * k];
    if (rok) Wm[i + n * j] = sacc;
  }
  __syncwarp(gmask);
  // ---- R = L_B^-1 W: lane i holds row i of L_B^-1; row i of R stays in registers
#pragma unroll
  for (int k = 0; k < NM; ++k) row[k] = (rok && k < n) ? LBi[gf + i + n * k] : (T)0;
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    T sacc = (T)0;
    if (j < n) {
#pragma unroll
      for (int k = 0; k < NM; ++k)
        if (k < n) sacc += row[k] * Wm[k + n * j];
    }
    acc[j] = sacc;
  }
  __syncwarp(gmask);
  // ---- T1 with its diagonal 1x1 / 2x2 blocks removed, and the block starts
  uint32_t cst = 0;
  {
    const uint32_t m1 = eok ? masks[2 * ef] : 0u;
    int r = 0;
    while (r < n) {
      const bool two = ((m1 >> r) & 1u) && r + 1 < n;
      if (two) cst |= 1u << r;
      r += two ? 2 : 1;
    }
  }
  if (eok)
    for (int q = i; q < nn; q += NM) {
      const int rr = q % n, c = q / n;
      const bool inblk = (rr == c) || (rr + 1 == c && ((cst >> rr) & 1u)) ||
                         (c + 1 == rr && ((cst >> c) & 1u));
      Fa[q] = inblk ? (T)0 : T1[gf + q];
    }
  __syncwarp(gmask);
  // ---- column sweep, last column first.  FP32: the rows of the next column's
  // inverses are loaded one column ahead (their addresses do not depend on the
  // sweep), so the global-load latency overlaps the current column's work.
  constexpr bool PF = sizeof(T) == 4 && NM <= 16;
  T rsave = (T)0;
  T cs[PF ? NM : 1], cp[PF ? NM : 1];
  if constexpr (PF) {
    const T* gs0 = Ge + (size_t)(2 * (n - 1)) * nn + (rok ? i : 0);
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      cs[k] = (k < n) ? gs0[(size_t)k * n] : (T)0;
      cp[k] = (k < n) ? gs0[nn + (size_t)k * n] : (T)0;
    }
  }
#pragma unroll
  for (int jj = NM - 1; jj >= 0; --jj) {
    if (jj < n) {
      const T r = acc[jj];
      const bool lo = ((cst >> jj) & 1u) != 0;                       // first column of a pair
      const bool up = jj >= 1 && ((cst >> (jj - 1)) & 1u) != 0;      // second column of a pair
      T rp = (T)0;
      if (up) rp = acc[jj >= 1 ? jj - 1 : 0];
      else if (lo) rp = rsave;
      if (rok) {
        Wm[i] = r;
        Wm[NM + i] = rp;
      }
      __syncwarp(gmask);
      T z0 = (T)0, z1 = (T)0;
      if constexpr (PF) {
        T ns[NM], np[NM];
        const T* gn = Ge + (size_t)(2 * (jj > 0 ? jj - 1 : 0)) * nn + (rok ? i : 0);
#pragma unroll
        for (int k = 0; k < NM; ++k) {
          ns[k] = (jj > 0 && k < n) ? gn[(size_t)k * n] : (T)0;
          np[k] = (jj > 0 && k < n) ? gn[nn + (size_t)k * n] : (T)0;
        }
#pragma unroll
        for (int k = 0; k < NM; k += 2) {
          if (k < n) z0 += cs[k] * Wm[k] + cp[k] * Wm[NM + k];
          if (k + 1 < n) z1 += cs[k + 1] * Wm[k + 1] + cp[k + 1] * Wm[NM + k + 1];
        }
#pragma unroll
        for (int k = 0; k < NM; ++k) {
          cs[k] = ns[k];
          cp[k] = np[k];
        }
      } else {
        const T* gs = Ge + (size_t)(2 * jj) * nn + (rok ? i : 0);   // idle lanes read row 0
#pragma unroll
        for (int k = 0; k < NM; k += 2) {
          if (k < n) z0 += gs[(size_t)k * n] * Wm[k];
          if (k + 1 < n) z1 += gs[(size_t)(k + 1) * n] * Wm[k + 1];
        }
        if (__any_sync(0xffffffffu, eok && (lo || up))) {
          const T* gp = gs + nn;
#pragma unroll
          for (int k = 0; k < NM; k += 2) {
            if (k < n) z0 += gp[(size_t)k * n] * Wm[NM + k];
            if (k + 1 < n) z1 += gp[(size_t)(k + 1) * n] * Wm[NM + k + 1];
          }
        }
      }
      const T z = z0 + z1;
      __syncwarp(gmask);
      rsave = r;
      acc[jj] = z;
#pragma unroll
      for (int jp = 0; jp < jj; ++jp) acc[jp] -= Fa[jp + n * jj] * z;
    }
  }
  __syncwarp(gmask);
  if (eok)
    for (int q = i; q < nn; q += NM) Fa[q] = Q1[gf + q];
  __syncwarp(gmask);
  // ---- x = Z Q1^T: lane i holds row i of Z (acc)
#pragma unroll
  for (int k = 0; k < NM; ++k) row[k] = (rok && k < n) ? acc[k] : (T)0;
  for (int j = 0; j < n; ++j) {
    T sacc = (T)0;
#pragma unroll
    for (int k = 0; k < NM; ++k)
      if (k < n) sacc += row[k] * Fa[j + n * k];
    if (rok) x[g + i + n * j] = (VT)sacc;
  }
}

template <typename T, int NM, typename VT>
cudaError_t launch_g(int n, int64_t E, const T* SA, const T* LBi, const T* Q1, const T* T1,
                     const T* G, const uint32_t* masks, const VT* b, VT* x,
                     const int32_t* skip, int fdiv, cudaStream_t s) {
  constexpr int EPW = 32 / NM;
  const int warps = 4;
  const int64_t per_block = (int64_t)warps * EPW;
  const int64_t blocks = (E + per_block - 1) / per_block;
  const size_t smem = (size_t)warps * EPW * 2 * NM * NM * sizeof(T);
  cudaError_t err = cudaFuncSetAttribute(k_apply_2d_g<T, NM, VT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_apply_2d_g<T, NM, VT><<<(unsigned)blocks, warps * 32, smem, s>>>(n, E, SA, LBi, Q1, T1, G,
                                                                      masks, b, x, skip, fdiv);
  count_launch();
  return cudaGetLastError();
}

template <typename T, int NM, typename VT>
cudaError_t launch_w(int n, int64_t E, const T* SA, const T* SB, const T* Q1, const T* Q2,
                     const T* T1, const T* T2, const uint32_t* masks, const VT* b, VT* x,
                     const int32_t* skip, int fdiv, cudaStream_t s) {
  constexpr int EPW = 32 / NM;
  const int warps = (NM == 32 && sizeof(T) == 8) ? 2 : 4;
  const int64_t per_block = (int64_t)warps * EPW;
  const int64_t blocks = (E + per_block - 1) / per_block;
  const size_t smem = (size_t)warps * EPW * 3 * NM * NM * sizeof(T) +
                      (size_t)warps * EPW * (3 * NM + 4) * sizeof(int);
  cudaError_t err = cudaFuncSetAttribute(k_apply_2d_w<T, NM, VT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_apply_2d_w<T, NM, VT><<<(unsigned)blocks, warps * 32, smem, s>>>(n, E, SA, SB, Q1, Q2, T1,
                                                                      T2, masks, b, x, skip, fdiv);
  count_launch();
  return cudaGetLastError();
}

template <typename T, typename VT>
cudaError_t launch_apply_one(const tpp_ctx* c, const T* SA, const T* LBi, const T* Q1,
                             const T* T1, const T* G, const VT* b, VT* x,
                             const int32_t* skip, cudaStream_t s) {
  const uint32_t* masks = c->p<uint32_t>(c->L.masks);
  // 2D blocks: vector blocks (E R), or their z slices in 3D; factors per element
  const int fdiv = ((c->dim == 3) ? c->n : 1) * c->R;
  const int64_t nb = c->EB * ((c->dim == 3) ? c->n : 1);
  if (c->n <= 8)
    return launch_g<T, 8, VT>(c->n, nb, SA, LBi, Q1, T1, G, masks, b, x, skip, fdiv, s);
  if (c->n <= 16)
    return launch_g<T, 16, VT>(c->n, nb, SA, LBi, Q1, T1, G, masks, b, x, skip, fdiv, s);
  return launch_g<T, 32, VT>(c->n, nb, SA, LBi, Q1, T1, G, masks, b, x, skip, fdiv, s);
}

template <typename T, typename VT>
cudaError_t launch_apply_t(const tpp_ctx* c, const T* SA, const T* SB, const T* Q1, const T* Q2,
                           const T* T1, const T* T2, const VT* b, VT* x,
                           const int32_t* skip, cudaStream_t s) {
  const uint32_t* masks = c->p<uint32_t>(c->L.masks);
  const int fdiv = ((c->dim == 3) ? c->n : 1) * c->R;
  const int64_t nb = c->EB * ((c->dim == 3) ? c->n : 1);   // 2D blocks (or z slices in 3D)
  if (c->n <= 8)
    return launch_w<T, 8, VT>(c->n, nb, SA, SB, Q1, Q2, T1, T2, masks, b, x, skip, fdiv, s);
  if (c->n <= 16)
    return launch_w<T, 16, VT>(c->n, nb, SA, SB, Q1, Q2, T1, T2, masks, b, x, skip, fdiv, s);
  return launch_w<T, 32, VT>(c->n, nb, SA, SB, Q1, Q2, T1, T2, masks, b, x, skip, fdiv, s);
}

template <typename VT>
cudaError_t launch_apply_2d_t(const tpp_ctx* c, const VT* b, VT* x, int prec,
                              const int32_t* skip, cudaStream_t s) {
  const bool two = two_sided(c);
  if (prec == TPP_FP64) {
    if (!two)
      return launch_apply_one<double, VT>(c, c->p<double>(c->L.fSA), c->p<double>(c->L.fSB),
                                          c->p<double>(c->L.fQ1), c->p<double>(c->L.fT1),
                                          c->p<double>(c->L.fG), b, x, skip, s);
    return launch_apply_t<double, VT>(c, c->p<double>(c->L.fSA), c->p<double>(c->L.fSB),
                                      c->p<double>(c->L.fQ1), c->p<double>(c->L.fQ2),
                                      c->p<double>(c->L.fT1), c->p<double>(c->L.fT2), b, x, skip,
                                      s);
  }
  const float* f = c->p<float>(c->L.f32);
  const F32Layout F = f32_layout(c->n, c->E, c->dim, two);
  if (!two)
    return launch_apply_one<float, VT>(c, f + F.SA, f + F.SB, f + F.Q1, f + F.T1, f + F.G, b, x,
                                       skip, s);
  return launch_apply_t<float, VT>(c, f + F.SA, f + F.SB, f + F.Q1, f + F.Q2, f + F.T1, f + F.T2,
                                   b, x, skip, s);
}

cudaError_t launch_apply_2d(const tpp_ctx* c, const double* b, double* x, int prec,
                            const int32_t* skip, cudaStream_t s) {
  return launch_apply_2d_t<double>(c, b, x, prec, skip, s);
}

// float copies of the apply factors, rounded to nearest (up to 8 segments)
struct F32Copy {
  const double* src[8];
  size_t dst[8], count[8];
  int nseg;
};

__global__ void k_to_f32(F32Copy cp, float* out) {
  for (int sg = 0; sg < cp.nseg; ++sg) {
    const double* src = cp.src[sg];
    float* dst = out + cp.dst[sg];
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < cp.count[sg];
         g += (size_t)gridDim.x * blockDim.x)
      dst[g] = __double2float_rn(src[g]);
  }
}

cudaError_t launch_to_f32(const tpp_ctx* c, cudaStream_t s) {
  const bool two = two_sided(c);
  const F32Layout F = f32_layout(c->n, c->E, c->dim, two);
  const size_t m = (size_t)c->E * c->n * c->n;
  F32Copy cp{};
  int k = 0;
  auto add = [&](size_t off, const double* src, size_t count) {
    cp.src[k] = src;
    cp.dst[k] = off;
    cp.count[k] = count;
    ++k;
  };
  add(F.SA, c->p<double>(c->L.fSA), m);
  add(F.SB, c->p<double>(c->L.fSB), m);
  add(F.Q1, c->p<double>(c->L.fQ1), m);
  add(F.T1, c->p<double>(c->L.fT1), m);
  if (two) {
    add(F.Q2, c->p<double>(c->L.fQ2), m);
    add(F.T2, c->p<double>(c->L.fT2), m);
  } else if (!(c->features & TPP_FEAT_F32_SHIFTS)) {   // else formed in FP32 by the build
    add(F.G, c->p<double>(c->L.fG), 2 * m * c->n);
  }
  if (c->dim == 3) add(F.Azi, c->p<double>(c->L.fAzi), m);
  cp.nseg = k;
  k_to_f32<<<152 * 4, 256, 0, s>>>(cp, c->p<float>(c->L.f32));
  count_launch();
  return cudaGetLastError();
}

// ---- 3D (Alg. 3d-apply): x = (A1^-1 (x) D1^-1) b.  The z factor acts first,
// x~ = (A1^-1 (x) I) b, one thread per z line (i, j) of an element with the
// line in registers; then the 2D apply of D1^-1 = (B1 (x) C1 + B2 (x) C2)^-1
// runs in place on each z slice (n slices per element share its factors).
template <typename T, int NZ, typename VT>
__global__ void __launch_bounds__(128)
k_apply_z(int n, int64_t E, const T* __restrict__ Azi, const VT* __restrict__ b,
          VT* __restrict__ x, const int32_t* skip, int R) {
  if (skip && *skip) return;
  __shared__ T az[4][NZ * NZ];
  const int nn = n * n, n3 = nn * n;
  const int sub = threadIdx.x >> 5;                      // one element per warp
  const int64_t e = (int64_t)blockIdx.x * 4 + sub;
  if (e >= E) return;
  const int lane = threadIdx.x & 31;
  for (int q = lane; q < nn; q += 32) az[sub][q] = Azi[(e / R) * nn + q];   // block e: element e / R
  __syncwarp();
  const VT* be = b + e * n3;
  VT* xe = x + e * n3;
  for (int q = lane; q < nn; q += 32) {
    T line[NZ];
#pragma unroll
    for (int k = 0; k < NZ; ++k) line[k] = (k < n) ? (T)be[q + (int64_t)nn * k] : (T)0;
#pragma unroll
    for (int k = 0; k < NZ; ++k) {
      if (k < n) {
        T sv = (T)0;
#pragma unroll
        for (int k2 = 0; k2 < NZ; ++k2)
          if (k2 < n) sv += az[sub][k + n * k2] * line[k2];
        xe[q + (int64_t)nn * k] = (VT)sv;
      }
    }
  }
}

template <typename VT>
cudaError_t launch_apply_3d_t(const tpp_ctx* c, const VT* b, VT* x, int prec,
                              const int32_t* skip, cudaStream_t s) {
  const int n = c->n;
  const unsigned blocks = (unsigned)((c->EB + 3) / 4);
  if (prec == TPP_FP64) {
    const double* azi = c->p<double>(c->L.fAzi);
    if (n <= 8) k_apply_z<double, 8, VT><<<blocks, 128, 0, s>>>(n, c->EB, azi, b, x, skip, c->R);
    else k_apply_z<double, 16, VT><<<blocks, 128, 0, s>>>(n, c->EB, azi, b, x, skip, c->R);
  } else {
    const float* azi = c->p<float>(c->L.f32) + f32_layout(n, c->E, 3, two_sided(c)).Azi;
    if (n <= 8) k_apply_z<float, 8, VT><<<blocks, 128, 0, s>>>(n, c->EB, azi, b, x, skip, c->R);
    else k_apply_z<float, 16, VT><<<blocks, 128, 0, s>>>(n, c->EB, azi, b, x, skip, c->R);
  }
  count_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  return launch_apply_2d_t<VT>(c, x, x, prec, skip, s);
}

cudaError_t launch_apply_3d(const tpp_ctx* c, const double* b, double* x, int prec,
                            const int32_t* skip, cudaStream_t s) {
  return launch_apply_3d_t<double>(c, b, x, prec, skip, s);
}

// FP32 factors, float vectors (the inner solves of the mixed-precision mode)
cudaError_t launch_apply_f32(const tpp_ctx* c, const float* b, float* x, const int32_t* skip,
                             cudaStream_t s) {
  if (c->dim == 2) return launch_apply_2d_t<float>(c, b, x, TPP_FP32, skip, s);
  return launch_apply_3d_t<float>(c, b, x, TPP_FP32, skip, s);
}

}  // namespace tpp
