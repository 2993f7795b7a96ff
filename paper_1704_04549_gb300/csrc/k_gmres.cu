// Krylov kernels for restarted right-preconditioned GMRES (Sec. 5 opening).
//
// Arnoldi uses classical Gram-Schmidt with one reorthogonalisation (CGS2):
// three streaming passes over the basis per step (dots, update+dots,
// update+norm), each reduced deterministically (fixed-order per-block
// partials, then one block sums them in block order).  Givens rotations and
// the least-squares back substitution run in one thread on the device.
#include "tpp_internal.cuh"

namespace tpp {

constexpr int kRedThreads = 256;
constexpr int kMaxBasis = 64;       // restart + 1 vectors at most

// partials[blk * stride + i] = sum over this block's slice of V_i . w, i < nvec
__device__ void dot_block(const double* __restrict__ V, int64_t N, int nvec,
                          const double* __restrict__ w, double* __restrict__ partials,
                          int stride, double* red) {
  for (int g0 = 0; g0 < nvec; g0 += 16) {
    const int gcount = (nvec - g0) < 16 ? (nvec - g0) : 16;
    double acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
         t += (int64_t)gridDim.x * blockDim.x) {
      const double wv = w[t];
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (i < gcount) acc[i] += V[(size_t)(g0 + i) * N + t] * wv;
    }
    // per-warp partial sums, then one warp per value folds the 8 warp sums
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      if (i < gcount) {
        const double v = warp_sum(acc[i]);
        if (lane == 0) red[i * 8 + wid] = v;
      }
    }
    __syncthreads();
    if (threadIdx.x < gcount) {
      double t = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[threadIdx.x * 8 + k];
      partials[blockIdx.x * stride + g0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// Last block of a grid: sum partials[b * stride + i] over all b (fixed order:
// lane-strided per warp, then a warp tree) into out[i] for i < nvec.
__device__ bool last_block(unsigned int* ticket) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  return is_last;
}

__device__ void final_reduce(const double* partials, int nblk, int stride, int nvec,
                             double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < nvec; i += nw) {
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += __ldcg(partials + (size_t)b * stride + i);
    s = warp_sum(s);
    if (lane == 0) out[i] = s;
  }
}

struct ArnoldiArgs {
  GmresState* st;
  double *H, *cs, *sn, *g, *h1, *h2, *inv_beta;
  int j;
};

// Close Arnoldi column j (single thread): H[0..j, j] = h1 + h2,
// H[j+1, j] = ||w||, previous Givens rotations, new rotation, g, flags.
// H is column-major (m+1) x m.
__device__ void finish_column(const ArnoldiArgs& a, double nrm2) {
  GmresState* st = a.st;
  const int m = st->m, j = a.j;
  const double hj1 = sqrt(nrm2);
  double* col = a.H + (size_t)j * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = a.h1[i] + a.h2[i];
  col[j + 1] = hj1;
  for (int i = 0; i < j; ++i) {
    const double t = a.cs[i] * col[i] + a.sn[i] * col[i + 1];
    col[i + 1] = -a.sn[i] * col[i] + a.cs[i] * col[i + 1];
    col[i] = t;
  }
  const double rho = hypot(col[j], col[j + 1]);
  double c = 1.0, s = 0.0;
  if (rho > 0.0) { c = col[j] / rho; s = col[j + 1] / rho; }
  a.cs[j] = c;
  a.sn[j] = s;
  col[j] = rho;
  col[j + 1] = 0.0;
  a.g[j + 1] = -s * a.g[j];
  a.g[j] = c * a.g[j];
  st->k = j + 1;
  st->est = fabs(a.g[j + 1]) / st->bnorm;
  *a.inv_beta = (hj1 > 0.0) ? 1.0 / hj1 : 0.0;
  if (!(hj1 > 0.0)) st->breakdown = 1;
  if (!(st->est == st->est)) st->breakdown = 2;
  if (st->est <= st->rtol || j + 1 >= m || st->breakdown) st->done = 1;
}

// pass 1 of CGS2: h1 = V^T w
__global__ void __launch_bounds__(kRedThreads)
k_dots(const double* V, int64_t N, int nvec, const double* w, double* partials, int stride,
       const int32_t* skip, double* h_out, unsigned int* ticket) {
  if (skip && *skip) return;
  __shared__ double red[16 * (kRedThreads / 32)];
  dot_block(V, N, nvec, w, partials, stride, red);
  if (last_block(ticket)) {
    final_reduce(partials, gridDim.x, stride, nvec, h_out);
    if (threadIdx.x == 0) *ticket = 0;
  }
}

// w -= V h_in; mode 0: h_out = V^T w (pass 2 of CGS2);
// mode 1: ||w||^2 and the Givens update of column a.j
__global__ void __launch_bounds__(kRedThreads)
k_update(const double* __restrict__ V, int64_t N, int nvec, const double* __restrict__ h_in,
         double* __restrict__ w, double* partials, int stride, int mode, const int32_t* skip,
         double* h_out, unsigned int* ticket, ArnoldiArgs aa) {
  if (skip && *skip) return;
  __shared__ double hs[kMaxBasis];
  __shared__ double red[16 * (kRedThreads / 32)];
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) hs[i] = h_in[i];
  __syncthreads();
  double nrm = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    double v = w[t];
    for (int i = 0; i < nvec; ++i) v -= hs[i] * V[(size_t)i * N + t];
    w[t] = v;
    nrm += v * v;
  }
  if (mode == 0) {
    __syncthreads();
    dot_block(V, N, nvec, w, partials, stride, red);
    if (last_block(ticket)) {
      final_reduce(partials, gridDim.x, stride, nvec, h_out);
      if (threadIdx.x == 0) *ticket = 0;
    }
  } else {
    const double s = block_sum(nrm, red);
    if (threadIdx.x == 0) partials[blockIdx.x * stride] = s;
    if (last_block(ticket)) {
      __shared__ double tot;
      final_reduce(partials, gridDim.x, stride, 1, &tot);
      __syncthreads();
      if (threadIdx.x == 0) {
        finish_column(aa, tot);
        *ticket = 0;
      }
    }
  }
}

// y = R^-1 g for the k x k upper-triangular part of the rotated H.  Single thread.
__global__ void k_lsq(const GmresState* st, const double* H, const double* g, double* y) {
  if (threadIdx.x != 0) return;
  const int k = st->k, m = st->m;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < k; ++l) s -= H[(size_t)l * (m + 1) + i] * y[l];
    const double d = H[(size_t)i * (m + 1) + i];
    y[i] = (d != 0.0) ? s / d : 0.0;
  }
}

// out = sum_{i < k} y_i B_i (+ out if accumulate)
__global__ void k_combine(const double* __restrict__ B, int64_t N, const GmresState* st,
                          const double* __restrict__ y, double* __restrict__ out, int accumulate) {
  __shared__ double ys[kMaxBasis];
  const int k = st->k;
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    double s = accumulate ? out[t] : 0.0;
    for (int i = 0; i < k; ++i) s += ys[i] * B[(size_t)i * N + t];
    out[t] = s;
  }
}

// y = a * x (+ b * y), scalars read from device memory when pointers given
__global__ void k_scale(double* __restrict__ out, const double* __restrict__ in, int64_t N,
                        const double* sptr, double sval, const int32_t* skip) {
  if (skip && *skip) return;
  const double sc = sptr ? *sptr : sval;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = sc * in[t];
}

__global__ void k_sub(double* __restrict__ out, const double* __restrict__ a,
                      const double* __restrict__ b, int64_t N) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = a[t] - b[t];
}

__global__ void __launch_bounds__(kRedThreads)
k_norm_partials(const double* __restrict__ x, int64_t N, double* partials, int stride) {
  __shared__ double red[kRedThreads / 32];
  double s = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    s += x[t] * x[t];
  s = block_sum(s, red);
  if (threadIdx.x == 0) partials[blockIdx.x * stride] = s;
}

__global__ void k_norm_finish(const double* partials, int nblk, int stride, double* out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partials[b * stride];
  *out = sqrt(s);
}

__global__ void k_cycle_init(GmresState* st, double* g, double beta, int m, double bnorm,
                             double rtol) {
  if (threadIdx.x != 0) return;
  st->bnorm = bnorm;
  st->rtol = rtol;
  st->est = beta / bnorm;
  st->j = 0;
  st->done = 0;
  st->k = 0;
  st->breakdown = 0;
  st->beta = beta;
  st->m = m;
  for (int i = 0; i <= m; ++i) g[i] = 0.0;
  g[0] = beta;
}

// ---------------------------------------------------------------------------
// launch helpers used by the host solver
cudaError_t gmres_dots(const double* V, int64_t N, int nvec, const double* w, double* partials,
                       int stride, int nblk, const int32_t* skip, double* h_out,
                       unsigned int* ticket, cudaStream_t s) {
  k_dots<<<nblk, kRedThreads, 0, s>>>(V, N, nvec, w, partials, stride, skip, h_out, ticket);
  count_launch();
  return cudaGetLastError();
}
cudaError_t gmres_update(const double* V, int64_t N, int nvec, const double* h, double* w,
                         double* partials, int stride, int mode, int nblk, const int32_t* skip,
                         double* h_out, unsigned int* ticket, GmresState* st, double* H,
                         double* cs, double* sn, double* g, double* h1, double* h2,
                         double* inv_beta, int j, cudaStream_t s) {
  ArnoldiArgs aa{st, H, cs, sn, g, h1, h2, inv_beta, j};
  k_update<<<nblk, kRedThreads, 0, s>>>(V, N, nvec, h, w, partials, stride, mode, skip, h_out,
                                        ticket, aa);
  count_launch();
  return cudaGetLastError();
}
cudaError_t gmres_lsq(const GmresState* st, const double* H, const double* g, double* y,
                      cudaStream_t s) {
  k_lsq<<<1, 32, 0, s>>>(st, H, g, y);
  count_launch();
  return cudaGetLastError();
}
cudaError_t gmres_combine(const double* B, int64_t N, const GmresState* st, const double* y,
                          double* out, int accumulate, cudaStream_t s) {
  k_combine<<<152 * 4, 256, 0, s>>>(B, N, st, y, out, accumulate);
  count_launch();
  return cudaGetLastError();
}
cudaError_t vec_scale(double* out, const double* in, int64_t N, const double* sptr, double sval,
                      const int32_t* skip, cudaStream_t s) {
  k_scale<<<152 * 4, 256, 0, s>>>(out, in, N, sptr, sval, skip);
  count_launch();
  return cudaGetLastError();
}
cudaError_t vec_sub(double* out, const double* a, const double* b, int64_t N, cudaStream_t s) {
  k_sub<<<152 * 4, 256, 0, s>>>(out, a, b, N);
  count_launch();
  return cudaGetLastError();
}
cudaError_t vec_norm(const double* x, int64_t N, double* partials, int stride, int nblk,
                     double* out, cudaStream_t s) {
  k_norm_partials<<<nblk, kRedThreads, 0, s>>>(x, N, partials, stride);
  count_launch();
  k_norm_finish<<<1, 32, 0, s>>>(partials, nblk, stride, out);
  count_launch();
  return cudaGetLastError();
}
cudaError_t gmres_cycle_init(GmresState* st, double* g, double beta, int m, double bnorm,
                             double rtol, cudaStream_t s) {
  k_cycle_init<<<1, 32, 0, s>>>(st, g, beta, m, bnorm, rtol);
  count_launch();
  return cudaGetLastError();
}

}  // namespace tpp

namespace tpp {

__global__ void k_axpy(double* __restrict__ out, const double* __restrict__ in, double a,
                       int64_t N) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] += a * in[t];
}

cudaError_t vec_axpy(double* out, const double* in, double a, int64_t N, cudaStream_t s) {
  k_axpy<<<152 * 4, 256, 0, s>>>(out, in, a, N);
  count_launch();
  return cudaGetLastError();
}

}  // namespace tpp
