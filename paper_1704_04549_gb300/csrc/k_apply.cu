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

constexpr int kApplyThreads = 256;

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

// Quasi-triangular Sylvester solve T2 Y + Y T1^T = C in shared memory
// (column-major, ld n; C is overwritten by Y), right-looking over the
// anti-diagonals of the 1x1 / 2x2 diagonal-block grid: block (I, J) sits on
// anti-diagonal (nbr - 1 - I) + (nbc - 1 - J).  At step s every block of that
// anti-diagonal is final, so (A) one thread per block solves its small
// system, then (B) every still-unsolved entry subtracts the contributions of
// the blocks solved at this step in its column (T2[i, k] Y[k, j]) and in its
// row (Y[i, l] T1[j, l]).  Each step has constant depth and phase B keeps all
// threads busy.  rowblk / colblk map a row / column to its block; rdiag holds
// 1 / (T2_ii + T1_jj) for the 1x1 solves.
template <typename T>
__device__ void sylvester_block(const T* T2, const T* T1, T* Y, int n, const int* rs,
                                const int* cs, int nbr, int nbc, const int* rowblk,
                                const int* colblk, const T* rdiag) {
  const int tid = threadIdx.x, nt = blockDim.x, nn = n * n;
  for (int s = 0; s < nbr + nbc - 1; ++s) {
    for (int a = tid; a < nbr; a += nt) {                    // (A) solve this anti-diagonal
      const int b = s - a;
      if (b < 0 || b >= nbc) continue;
      const int I = nbr - 1 - a, J = nbc - 1 - b;
      const int i0 = rs[I], ni = rs[I + 1] - i0, j0 = cs[J], nj = cs[J + 1] - j0;
      if (ni == 1 && nj == 1) {
        Y[i0 + n * j0] *= rdiag[i0 + n * j0];
      } else {
        T ab[4] = {(T)0, (T)0, (T)0, (T)0}, bb[4] = {(T)0, (T)0, (T)0, (T)0};
        T rhs[4] = {(T)0, (T)0, (T)0, (T)0};
        ab[0] = T2[i0 + n * i0];
        bb[0] = T1[j0 + n * j0];
        rhs[0] = Y[i0 + n * j0];
        if (ni == 2) {
          ab[1] = T2[(i0 + 1) + n * i0];
          ab[2] = T2[i0 + n * (i0 + 1)];
          ab[3] = T2[(i0 + 1) + n * (i0 + 1)];
          rhs[1] = Y[(i0 + 1) + n * j0];
        }
        if (nj == 2) {
          bb[1] = T1[(j0 + 1) + n * j0];
          bb[2] = T1[j0 + n * (j0 + 1)];
          bb[3] = T1[(j0 + 1) + n * (j0 + 1)];
          rhs[ni] = Y[i0 + n * (j0 + 1)];
        }
        if (ni == 2 && nj == 2) rhs[3] = Y[(i0 + 1) + n * (j0 + 1)];
        small_sylvester<T>(ni, nj, ab, bb, rhs);
        Y[i0 + n * j0] = rhs[0];
        if (ni == 2) Y[(i0 + 1) + n * j0] = rhs[1];
        if (nj == 2) Y[i0 + n * (j0 + 1)] = rhs[ni];
        if (ni == 2 && nj == 2) Y[(i0 + 1) + n * (j0 + 1)] = rhs[3];
      }
    }
    __syncthreads();
    if (s + 1 < nbr + nbc - 1) {                               // (B) rank updates
      for (int q = tid; q < nn; q += nt) {
        const int i = q % n, j = q / n;
        const int I = rowblk[i], J = colblk[j];
        if ((nbr - 1 - I) + (nbc - 1 - J) <= s) continue;      // solved already
        T v = (T)0;
        const int a = s - (nbc - 1 - J);                        // block solved in column J
        if (a >= 0 && a < nbr) {
          const int Is = nbr - 1 - a;
          for (int k = rs[Is]; k < rs[Is + 1]; ++k) v += T2[i + n * k] * Y[k + n * j];
        }
        const int b = s - (nbr - 1 - I);                        // block solved in row I
        if (b >= 0 && b < nbc) {
          const int Js = nbc - 1 - b;
          for (int l = cs[Js]; l < cs[Js + 1]; ++l) v += Y[i + n * l] * T1[j + n * l];
        }
        Y[q] -= v;
      }
      __syncthreads();
    }
  }
}

__device__ int blocks_from_mask(uint32_t mask, int n, int* starts, int* blk) {
  int nb = 0, i = 0;
  while (i < n) {
    starts[nb] = i;
    const int w = ((mask >> i) & 1u) && (i + 1 < n) ? 2 : 1;
    for (int t = 0; t < w; ++t) blk[i + t] = nb;
    ++nb;
    i += w;
  }
  starts[nb] = n;
  return nb;
}

}  // namespace

// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kApplyThreads)
k_apply_2d(int n, const T* __restrict__ SA, const T* __restrict__ SB, const T* __restrict__ Q1,
           const T* __restrict__ Q2, const T* __restrict__ T1, const T* __restrict__ T2,
           const uint32_t* __restrict__ masks, const double* __restrict__ b,
           double* __restrict__ x, const int32_t* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int nn = n * n;
  T* F0 = sm;           // factor buffer 0
  T* F1 = F0 + nn;      // factor buffer 1
  T* W0 = F1 + nn;      // work
  T* W1 = W0 + nn;      // work
  __shared__ int rs[TPP_MAX_N + 1], cs[TPP_MAX_N + 1];
  __shared__ int rowblk[TPP_MAX_N], colblk[TPP_MAX_N];
  __shared__ int nb[2];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t e = blockIdx.x;
  const int64_t base = e * nn;
  for (int q = tid; q < nn; q += nt) {
    F0[q] = SA[base + q];
    F1[q] = SB[base + q];
    W0[q] = (T)b[base + q];
  }
  if (tid == 0) nb[0] = blocks_from_mask(masks[2 * e + 1], n, rs, rowblk);   // T2 -> rows
  if (tid == 32) nb[1] = blocks_from_mask(masks[2 * e], n, cs, colblk);      // T1 -> columns
  __syncthreads();
  // W1 = B S_A^T
  for (int q = tid; q < nn; q += nt) {
    const int i = q % n, j = q / n;
    T s = (T)0;
    for (int k = 0; k < n; ++k) s += W0[i + n * k] * F0[j + n * k];
    W1[q] = s;
  }
  __syncthreads();
  // W0 = S_B W1   (= C)
  for (int q = tid; q < nn; q += nt) {
    const int i = q % n, j = q / n;
    T s = (T)0;
    for (int k = 0; k < n; ++k) s += F1[i + n * k] * W1[k + n * j];
    W0[q] = s;
  }
  __syncthreads();
  for (int q = tid; q < nn; q += nt) {
    F0[q] = T1[base + q];
    F1[q] = T2[base + q];
  }
  __syncthreads();
  // reciprocals of the 1x1 block denominators T2_ii + T1_jj, all lanes busy
  for (int q = tid; q < nn; q += nt) {
    const int i = q % n, j = q / n;
    W1[q] = (T)1 / (F1[i + n * i] + F0[j + n * j]);
  }
  __syncthreads();
  sylvester_block<T>(F1, F0, W0, n, rs, cs, nb[0], nb[1], rowblk, colblk, W1);   // W0 = Y
  __syncthreads();
  for (int q = tid; q < nn; q += nt) {
    F0[q] = Q1[base + q];
    F1[q] = Q2[base + q];
  }
  __syncthreads();
  // W1 = Y Q1^T
  for (int q = tid; q < nn; q += nt) {
    const int i = q % n, j = q / n;
    T s = (T)0;
    for (int k = 0; k < n; ++k) s += W0[i + n * k] * F0[j + n * k];
    W1[q] = s;
  }
  __syncthreads();
  // x = Q2 W1
  for (int q = tid; q < nn; q += nt) {
    const int i = q % n, j = q / n;
    T s = (T)0;
    for (int k = 0; k < n; ++k) s += F1[i + n * k] * W1[k + n * j];
    x[base + q] = (double)s;
  }
}

cudaError_t launch_apply_2d(const tpp_ctx* c, const double* b, double* x, int prec,
                            const int32_t* skip, cudaStream_t s) {
  const int n = c->n, nn = n * n;
  const uint32_t* masks = c->p<uint32_t>(c->L.masks);
  if (prec == TPP_FP64) {
    const size_t smem = 4 * (size_t)nn * sizeof(double);
    k_apply_2d<double><<<(unsigned)c->E, kApplyThreads, smem, s>>>(
        n, c->p<double>(c->L.fSA), c->p<double>(c->L.fSB), c->p<double>(c->L.fQ1),
        c->p<double>(c->L.fQ2), c->p<double>(c->L.fT1), c->p<double>(c->L.fT2), masks, b, x,
        skip);
    count_launch();
  } else {
    const size_t smem = 4 * (size_t)nn * sizeof(float);
    const float* f = c->p<float>(c->L.f32);
    const size_t st = (size_t)c->E * nn;
    k_apply_2d<float><<<(unsigned)c->E, kApplyThreads, smem, s>>>(
        n, f, f + st, f + 2 * st, f + 3 * st, f + 4 * st, f + 5 * st, masks, b, x, skip);
    count_launch();
  }
  return cudaGetLastError();
}

// float copies of the apply factors (SA, SB, Q1, Q2, T1, T2), rounded to nearest
__global__ void k_to_f32(const double* SA, const double* SB, const double* Q1, const double* Q2,
                         const double* T1, const double* T2, float* out, int64_t st) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < 6 * st;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int which = (int)(g / st);
    const int64_t i = g % st;
    const double* src = which == 0 ? SA : which == 1 ? SB : which == 2 ? Q1 : which == 3 ? Q2
                      : which == 4 ? T1 : T2;
    out[g] = __double2float_rn(src[i]);
  }
}

cudaError_t launch_to_f32(const tpp_ctx* c, cudaStream_t s) {
  const int64_t st = c->E * (int64_t)c->n * c->n;
  k_to_f32<<<152 * 4, 256, 0, s>>>(c->p<double>(c->L.fSA), c->p<double>(c->L.fSB),
                                   c->p<double>(c->L.fQ1), c->p<double>(c->L.fQ2),
                                   c->p<double>(c->L.fT1), c->p<double>(c->L.fT2),
                                   c->p<float>(c->L.f32), st);
  count_launch();
  return cudaGetLastError();
}

}  // namespace tpp
