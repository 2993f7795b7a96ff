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

// Solve (I (x) A + Bt (x) I) vec(Y) = vec(R) for a ni x nj block, ni, nj <= 2,
// A = T2 block (ni x ni), Bt = T1 block (nj x nj), column-major vec.  Gaussian
// elimination with partial pivoting on the <= 4 x 4 system.
template <typename T>
__device__ void small_sylvester(int ni, int nj, const T a[4], const T bt[4], T y[4]) {
  const int m = ni * nj;
  T Ms[4][5];
  for (int p = 0; p < m; ++p)
    for (int q = 0; q <= m; ++q) Ms[p][q] = (q == m) ? y[p] : (T)0;
  // vec index p = r + ni c  (r row in block, c column in block)
  for (int p = 0; p < m; ++p) {
    const int r = p % ni, c = p / ni;
    for (int q = 0; q < m; ++q) {
      const int r2 = q % ni, c2 = q / ni;
      T v = (T)0;
      if (c == c2) v += a[r + 2 * r2];          // A[r, r2]
      if (r == r2) v += bt[c + 2 * c2];         // Bt[c, c2]  (T1 block)
      Ms[p][q] = v;
    }
  }
  for (int k = 0; k < m; ++k) {
    int pr = k;
    for (int i = k + 1; i < m; ++i)
      if (fabs((double)Ms[i][k]) > fabs((double)Ms[pr][k])) pr = i;
    if (pr != k)
      for (int q = 0; q <= m; ++q) { T t = Ms[k][q]; Ms[k][q] = Ms[pr][q]; Ms[pr][q] = t; }
    const T piv = Ms[k][k];
    for (int i = k + 1; i < m; ++i) {
      const T f = Ms[i][k] / piv;
      for (int q = k; q <= m; ++q) Ms[i][q] -= f * Ms[k][q];
    }
  }
  for (int k = m - 1; k >= 0; --k) {
    T s = Ms[k][m];
    for (int q = k + 1; q < m; ++q) s -= Ms[k][q] * y[q];
    y[k] = s / Ms[k][k];
  }
}

// Wavefront quasi-triangular Sylvester solve T2 Y + Y T1^T = C in shared
// memory (column-major, ld n).  C is overwritten by Y.  rs/cs: block starts
// (ascending) of T2 rows / T1 columns, nbr/nbc their counts; blocks of size
// 2 start where the mask bit is set.
template <typename T>
__device__ void sylvester_wavefront(const T* T2, const T* T1, T* Y, int n, const int* rs,
                                    const int* cs, int nbr, int nbc) {
  const int tid = threadIdx.x;
  for (int s = 0; s < nbr + nbc - 1; ++s) {
    for (int a = tid; a < nbr; a += blockDim.x) {
      const int b = s - a;
      if (b < 0 || b >= nbc) continue;
      const int I = nbr - 1 - a, J = nbc - 1 - b;
      const int i0 = rs[I], ni = rs[I + 1] - i0;
      const int j0 = cs[J], nj = cs[J + 1] - j0;
      T rhs[4], ab[4], bb[4];
      for (int cc = 0; cc < nj; ++cc)
        for (int rr = 0; rr < ni; ++rr) {
          const int i = i0 + rr, j = j0 + cc;
          T v = Y[i + n * j];
          for (int k = i0 + ni; k < n; ++k) v -= T2[i + n * k] * Y[k + n * j];
          for (int l = j0 + nj; l < n; ++l) v -= Y[i + n * l] * T1[j + n * l];
          rhs[rr + ni * cc] = v;
        }
      for (int rr = 0; rr < ni; ++rr)
        for (int r2 = 0; r2 < ni; ++r2) ab[rr + 2 * r2] = T2[(i0 + rr) + n * (i0 + r2)];
      for (int c1 = 0; c1 < nj; ++c1)
        for (int c2 = 0; c2 < nj; ++c2) bb[c1 + 2 * c2] = T1[(j0 + c1) + n * (j0 + c2)];
      small_sylvester<T>(ni, nj, ab, bb, rhs);
      for (int cc = 0; cc < nj; ++cc)
        for (int rr = 0; rr < ni; ++rr) Y[(i0 + rr) + n * (j0 + cc)] = rhs[rr + ni * cc];
    }
    __syncthreads();
  }
}

__device__ int blocks_from_mask(uint32_t mask, int n, int* starts) {
  int nb = 0, i = 0;
  while (i < n) {
    starts[nb++] = i;
    i += ((mask >> i) & 1u) && (i + 1 < n) ? 2 : 1;
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
  __shared__ int nb[2];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t e = blockIdx.x;
  const int64_t base = e * nn;
  for (int q = tid; q < nn; q += nt) {
    F0[q] = SA[base + q];
    F1[q] = SB[base + q];
    W0[q] = (T)b[base + q];
  }
  if (tid == 0) nb[0] = blocks_from_mask(masks[2 * e + 1], n, rs);   // T2 -> rows
  if (tid == 32) nb[1] = blocks_from_mask(masks[2 * e], n, cs);      // T1 -> columns
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
  sylvester_wavefront<T>(F1, F0, W0, n, rs, cs, nb[0], nb[1]);   // W0 = Y
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
