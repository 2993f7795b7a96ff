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

constexpr int kRegBasis = 32;      // basis sizes kept in register tiles
constexpr int kWarps = kRedThreads / 32;

// Per-thread accumulators acc[i < cnt] -> partials[blk * stride + g0 + i]
// (deterministic).  Within a warp the G sums are formed by recursive halving:
// at each butterfly level a lane keeps half of its values and adds the
// partner's copy of them, so the warp issues G - 1 + (5 - log2 G) additions in
// total instead of 5 G for G separate shuffle trees (the additions are FP64
// instructions for double accumulators, a scarce pipe on this GPU).  Lane l
// ends with the value whose index is given by its bits 4, 3, ... (high to low);
// the warps' results are then added in warp order.
template <typename AT, int G>
__device__ void store_block_partials(AT (&acc)[G], int cnt, int g0, double* partials,
                                     int stride, double* red) {
  static_assert(G == 8 || G == 16 || G == 32, "group size");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int LG = (G == 8) ? 3 : (G == 16) ? 4 : 5;
#pragma unroll
  for (int lev = 0; lev < LG; ++lev) {
    const int sft = 16 >> lev;                 // partner distance
    const int half = G >> (lev + 1);           // values kept per lane after this level
    const bool up = (lane & sft) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const AT send = up ? acc[k] : acc[k + half];
      const AT keep = up ? acc[k + half] : acc[k];
      acc[k] = keep + __shfl_xor_sync(0xffffffffu, send, sft);
    }
  }
#pragma unroll
  for (int sft = (16 >> LG); sft > 0; sft >>= 1) acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], sft);
  int idx = 0;
#pragma unroll
  for (int lev = 0; lev < LG; ++lev) idx = 2 * idx + ((lane >> (4 - lev)) & 1);
  if ((lane & ((1 << (5 - LG)) - 1)) == 0 && idx < cnt) red[idx * kWarps + wid] = (double)acc[0];
  __syncthreads();
  if (threadIdx.x < cnt) {
    double t = 0.0;
    for (int k = 0; k < kWarps; ++k) t += red[threadIdx.x * kWarps + k];
    partials[blockIdx.x * stride + g0 + threadIdx.x] = t;
  }
  __syncthreads();
}

// block sum of one value in the accumulator type (float sums stay on the FMA pipe)
template <typename AT>
__device__ AT block_sum_t(AT v, AT* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  AT t = (AT)0;
  for (int k = 0; k < kWarps; ++k) t += red[k];
  __syncthreads();
  return t;
}

// partials of V_i . w for g0 <= i < g0 + cnt, cnt <= G.  The G loads of a point
// are issued unconditionally (indices past cnt repeat the last vector, a cache
// hit) so that they are all in flight together.
template <typename VT, int G>
__device__ void dot_group(const VT* __restrict__ V, int64_t N, int g0, int cnt,
                          const VT* __restrict__ w, double* __restrict__ partials, int stride,
                          double* red) {
  VT acc[G];
#pragma unroll
  for (int i = 0; i < G; ++i) acc[i] = (VT)0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    const VT wv = w[t];
    VT vv[G];
#pragma unroll
    for (int i = 0; i < G; ++i) vv[i] = V[(size_t)(g0 + (i < cnt ? i : cnt - 1)) * N + t];
#pragma unroll
    for (int i = 0; i < G; ++i) acc[i] += vv[i] * wv;
  }
  store_block_partials<VT, G>(acc, cnt, g0, partials, stride, red);
}

template <typename VT>
__device__ void dot_block(const VT* __restrict__ V, int64_t N, int nvec,
                          const VT* __restrict__ w, double* __restrict__ partials, int stride,
                          double* red) {
  for (int g0 = 0; g0 < nvec; g0 += kRegBasis) {
    const int cnt = (nvec - g0) < kRegBasis ? (nvec - g0) : kRegBasis;
    if (cnt <= 8) dot_group<VT, 8>(V, N, g0, cnt, w, partials, stride, red);
    else if (cnt <= 16) dot_group<VT, 16>(V, N, g0, cnt, w, partials, stride, red);
    else dot_group<VT, 32>(V, N, g0, cnt, w, partials, stride, red);
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
template <typename VT, int G>
__global__ void __launch_bounds__(kRedThreads)
k_dots(const VT* V, int64_t N, int nvec, const VT* w, double* partials, int stride,
       const int32_t* skip, double* h_out, unsigned int* ticket) {
  if (skip && *skip) return;
  __shared__ double red[kRegBasis * kWarps];
  if (G > 0) dot_group<VT, (G > 0 ? G : 8)>(V, N, 0, nvec, w, partials, stride, red);
  else dot_block(V, N, nvec, w, partials, stride, red);
  if (last_block(ticket)) {
    final_reduce(partials, gridDim.x, stride, nvec, h_out);
    if (threadIdx.x == 0) *ticket = 0;
  }
}

// w -= V h for one point per thread, nvec <= G vectors (loads unconditional,
// coefficients of the padded entries are zero); mode 0 also accumulates the
// products of the same basis entries with the updated w (pass 2 of CGS2 in one
// read of the basis), mode 1 the squared norm.
template <typename VT, int G>
__device__ void update_group(const VT* __restrict__ V, int64_t N, int nvec, const VT* hs,
                             VT* __restrict__ w, int mode, VT& nrm, double* partials,
                             int stride, double* red) {
  VT acc[G];
#pragma unroll
  for (int i = 0; i < G; ++i) acc[i] = (VT)0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    VT vv[G];
#pragma unroll
    for (int i = 0; i < G; ++i) vv[i] = V[(size_t)(i < nvec ? i : nvec - 1) * N + t];
    VT wv = w[t];
#pragma unroll
    for (int i = 0; i < G; ++i) wv -= hs[i] * vv[i];
    w[t] = wv;
    if (mode == 0) {
#pragma unroll
      for (int i = 0; i < G; ++i) acc[i] += vv[i] * wv;
    } else {
      nrm += wv * wv;
    }
  }
  if (mode == 0) store_block_partials<VT, G>(acc, nvec, 0, partials, stride, red);
}

// w -= V h_in; mode 0: h_out = V^T w (pass 2 of CGS2, fused: the basis entries
// of a point stay in registers for both products when nvec <= kRegBasis);
// mode 1: ||w||^2 and the Givens update of column a.j; mode 2 (first pass of
// the selectively reorthogonalised Gram-Schmidt): ||w||^2, and if it kept at
// least half of ||w_before||^2 = h_in[nvec] (the norm did not drop by more than
// 1/sqrt 2: Daniel-Gragg-Kaufman-Stewart) the column is final, h2 = 0 and the
// Givens update runs here, st->skip_re = 1; otherwise st->skip_re = 0 and the
// second pass follows.  A skipped mode-2 launch sets skip_re = 1.
template <typename VT, int G>
__global__ void __launch_bounds__(kRedThreads)
k_update(const VT* __restrict__ V, int64_t N, int nvec, const double* __restrict__ h_in,
         VT* __restrict__ w, double* partials, int stride, int mode, const int32_t* skip,
         double* h_out, unsigned int* ticket, ArnoldiArgs aa) {
  if (skip && *skip) {
    if (mode == 2 && blockIdx.x == 0 && threadIdx.x == 0) aa.st->skip_re = 1;
    return;
  }
  __shared__ VT hs[kMaxBasis];
  __shared__ double red[kRegBasis * kWarps];
  for (int i = threadIdx.x; i < kMaxBasis; i += blockDim.x) hs[i] = (i < nvec) ? (VT)h_in[i] : (VT)0;
  __syncthreads();
  VT nrm = (VT)0;
  if (G > 0) {
    update_group<VT, (G > 0 ? G : 8)>(V, N, nvec, hs, w, mode, nrm, partials, stride, red);
  } else {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
         t += (int64_t)gridDim.x * blockDim.x) {
      VT v = w[t];
      for (int i = 0; i < nvec; ++i) v -= hs[i] * V[(size_t)i * N + t];
      w[t] = v;
      nrm += v * v;
    }
    if (mode == 0) {
      __syncthreads();
      dot_block(V, N, nvec, w, partials, stride, red);
    }
  }
  if (mode == 0) {
    if (last_block(ticket)) {
      final_reduce(partials, gridDim.x, stride, nvec, h_out);
      if (threadIdx.x == 0) *ticket = 0;
    }
  } else {
    const double sblk = (double)block_sum_t<VT>(nrm, reinterpret_cast<VT*>(red));
    if (threadIdx.x == 0) partials[blockIdx.x * stride] = sblk;
    if (last_block(ticket)) {
      __shared__ double tot;
      final_reduce(partials, gridDim.x, stride, 1, &tot);
      __syncthreads();
      if (threadIdx.x == 0) {
        if (mode == 1) {
          finish_column(aa, tot);
        } else if (tot >= 0.5 * h_in[nvec]) {
          for (int i = 0; i < nvec; ++i) aa.h2[i] = 0.0;
          finish_column(aa, tot);
          aa.st->skip_re = 1;
        } else {
          aa.st->skip_re = 0;
        }
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
template <typename VI, typename VO>
__global__ void k_combine(const VI* __restrict__ B, int64_t N, const GmresState* st,
                          const double* __restrict__ y, VO* __restrict__ out, int accumulate,
                          const int32_t* skip) {
  if (skip && *skip) return;
  __shared__ VI ys[kMaxBasis];
  const int k = st->k;
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = (VI)y[i];
  __syncthreads();
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    VI s = (VI)0;
    for (int i = 0; i < k; ++i) s += ys[i] * B[(size_t)i * N + t];
    out[t] = accumulate ? (VO)(out[t] + (VO)s) : (VO)s;
  }
}

// out = sc * in, sc read from device memory when sptr is given
template <typename VT>
__global__ void k_scale(VT* __restrict__ out, const VT* __restrict__ in, int64_t N,
                        const double* sptr, double sval, const int32_t* skip) {
  if (skip && *skip) return;
  const VT sc = (VT)(sptr ? *sptr : sval);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = sc * in[t];
}

// float copy of a vector (rounded to nearest)
__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, int64_t N,
                           const int32_t* skip) {
  if (skip && *skip) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = __double2float_rn(in[t]);
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
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 32) s += partials[b * stride];
  s = warp_sum(s);
  if (threadIdx.x == 0) *out = sqrt(s);
}

__global__ void k_cycle_init(GmresState* st, double* g, double beta, int m, double bnorm,
                             double rtol, const int32_t* done_src) {
  if (threadIdx.x != 0) return;
  st->bnorm = bnorm;
  st->rtol = rtol;
  st->est = beta / bnorm;
  st->j = 0;
  st->done = done_src ? *done_src : 0;
  st->k = 0;
  st->breakdown = 0;
  st->beta = beta;
  st->m = m;
  for (int i = 0; i <= m; ++i) g[i] = 0.0;
  g[0] = beta;
}

// ---------------------------------------------------------------------------
// launch helpers used by the host solver (VT = double: the FP64 solver, float:
// the inner solves of the mixed-precision mode)
constexpr int kVecBlocks = 152 * 4;     // grid of the basis kernels

template <typename VT>
cudaError_t gmres_dots(const VT* V, int64_t N, int nvec, const VT* w, double* partials,
                       int stride, int nblk, const int32_t* skip, double* h_out,
                       unsigned int* ticket, cudaStream_t s) {
  const int g = nblk < kVecBlocks ? nblk : kVecBlocks;
  if (nvec <= 8)
    k_dots<VT, 8><<<g, kRedThreads, 0, s>>>(V, N, nvec, w, partials, stride, skip, h_out, ticket);
  else if (nvec <= 16)
    k_dots<VT, 16><<<g, kRedThreads, 0, s>>>(V, N, nvec, w, partials, stride, skip, h_out, ticket);
  else if (nvec <= kRegBasis)
    k_dots<VT, 32><<<g, kRedThreads, 0, s>>>(V, N, nvec, w, partials, stride, skip, h_out, ticket);
  else
    k_dots<VT, 0><<<g, kRedThreads, 0, s>>>(V, N, nvec, w, partials, stride, skip, h_out, ticket);
  count_launch();
  return cudaGetLastError();
}
template <typename VT>
cudaError_t gmres_update(const VT* V, int64_t N, int nvec, const double* h, VT* w,
                         double* partials, int stride, int mode, int nblk, const int32_t* skip,
                         double* h_out, unsigned int* ticket, GmresState* st, double* H,
                         double* cs, double* sn, double* g, double* h1, double* h2,
                         double* inv_beta, int j, cudaStream_t s) {
  ArnoldiArgs aa{st, H, cs, sn, g, h1, h2, inv_beta, j};
  const int gr = nblk < kVecBlocks ? nblk : kVecBlocks;
  if (nvec <= 8)
    k_update<VT, 8><<<gr, kRedThreads, 0, s>>>(V, N, nvec, h, w, partials, stride, mode, skip,
                                               h_out, ticket, aa);
  else if (nvec <= 16)
    k_update<VT, 16><<<gr, kRedThreads, 0, s>>>(V, N, nvec, h, w, partials, stride, mode, skip,
                                                h_out, ticket, aa);
  else if (nvec <= kRegBasis)
    k_update<VT, 32><<<gr, kRedThreads, 0, s>>>(V, N, nvec, h, w, partials, stride, mode, skip,
                                                h_out, ticket, aa);
  else
    k_update<VT, 0><<<gr, kRedThreads, 0, s>>>(V, N, nvec, h, w, partials, stride, mode, skip,
                                               h_out, ticket, aa);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t gmres_dots<double>(const double*, int64_t, int, const double*, double*, int,
                                        int, const int32_t*, double*, unsigned int*, cudaStream_t);
template cudaError_t gmres_dots<float>(const float*, int64_t, int, const float*, double*, int,
                                       int, const int32_t*, double*, unsigned int*, cudaStream_t);
template cudaError_t gmres_update<double>(const double*, int64_t, int, const double*, double*,
                                          double*, int, int, int, const int32_t*, double*,
                                          unsigned int*, GmresState*, double*, double*, double*,
                                          double*, double*, double*, double*, int, cudaStream_t);
template cudaError_t gmres_update<float>(const float*, int64_t, int, const double*, float*,
                                         double*, int, int, int, const int32_t*, double*,
                                         unsigned int*, GmresState*, double*, double*, double*,
                                         double*, double*, double*, double*, int, cudaStream_t);
cudaError_t gmres_lsq(const GmresState* st, const double* H, const double* g, double* y,
                      cudaStream_t s) {
  k_lsq<<<1, 32, 0, s>>>(st, H, g, y);
  count_launch();
  return cudaGetLastError();
}
cudaError_t gmres_combine(const double* B, int64_t N, const GmresState* st, const double* y,
                          double* out, int accumulate, cudaStream_t s) {
  k_combine<double, double><<<152 * 4, 256, 0, s>>>(B, N, st, y, out, accumulate, nullptr);
  count_launch();
  return cudaGetLastError();
}
cudaError_t gmres_combine_f32(const float* B, int64_t N, const GmresState* st, const double* y,
                              double* out, const int32_t* skip, cudaStream_t s) {
  k_combine<float, double><<<152 * 4, 256, 0, s>>>(B, N, st, y, out, 0, skip);
  count_launch();
  return cudaGetLastError();
}
cudaError_t vec_scale(double* out, const double* in, int64_t N, const double* sptr, double sval,
                      const int32_t* skip, cudaStream_t s) {
  k_scale<double><<<152 * 4, 256, 0, s>>>(out, in, N, sptr, sval, skip);
  count_launch();
  return cudaGetLastError();
}
cudaError_t vec_scale_f32(float* out, const float* in, int64_t N, const double* sptr,
                          double sval, const int32_t* skip, cudaStream_t s) {
  k_scale<float><<<152 * 4, 256, 0, s>>>(out, in, N, sptr, sval, skip);
  count_launch();
  return cudaGetLastError();
}
cudaError_t vec_to_float(const double* in, float* out, int64_t N, const int32_t* skip,
                         cudaStream_t s) {
  k_to_float<<<152 * 4, 256, 0, s>>>(in, out, N, skip);
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
                             double rtol, const int32_t* done_src, cudaStream_t s) {
  k_cycle_init<<<1, 32, 0, s>>>(st, g, beta, m, bnorm, rtol, done_src);
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

__global__ void k_accum_inner(GmresState* outer, const GmresState* inner, const int32_t* skip) {
  if (threadIdx.x == 0 && !(skip && *skip)) outer->inner_total += inner->k;
}

cudaError_t accumulate_inner(GmresState* outer, const GmresState* inner, const int32_t* skip,
                             cudaStream_t s) {
  k_accum_inner<<<1, 32, 0, s>>>(outer, inner, skip);
  count_launch();
  return cudaGetLastError();
}

cudaError_t vec_axpy(double* out, const double* in, double a, int64_t N, cudaStream_t s) {
  k_axpy<<<152 * 4, 256, 0, s>>>(out, in, a, N);
  count_launch();
  return cudaGetLastError();
}

}  // namespace tpp
