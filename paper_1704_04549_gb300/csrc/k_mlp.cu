// Learned Kronecker factors: an MLP that predicts an element's rank-2 factors
// from its velocity samples, its training kernels, and the factor build that
// uses the predictions with the exact KSVD as fallback.
//
// Network: 2 n^2 + 1 inputs (a_x, a_y at the n x n nodes, dt / h), three hidden
// layers of width 512 with the exact GELU, 4 n^2 outputs read as vec(A_1),
// vec(B_1), vec(A_2), vec(B_2) of the rearranged block scaled to unit Frobenius
// norm.  Weights are kept as FP32 master copies and used as BF16; every product
// accumulates in FP32.  Loss of an element (gauge invariant, Sec. 4.1 Eq. NKP):
//   L = || A~ / ||A~|| - sum_k a_k b_k^T ||_F^2,  a_k = vec(A_k), b_k = vec(B_k),
// evaluated through the structure A~ = Q M Q^T (Q = [E | Qo] orthonormal, M the
// r x r core) as L = 1 - 2 sum_k (Q^T a_k)^T Mn (Q^T b_k) + sum_kl (a_k.a_l)(b_k.b_l)
// with Mn = M / ||M||_F.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>

#include "tpp_internal.cuh"

struct tpp_mlp {
  int32_t n, max_batch;
  int32_t widths[5];
  int64_t woff[4], boff[4], nparams;   // offsets (floats) of W_l [K][N] row-major and b_l
  int64_t wbf_off[4];                   // offsets (bf16) of the BF16 weights
  char* ws;
  size_t ws_bytes;
  size_t p32, pbf, grad, am, av, act, pre, g0, g1, lossv, scal;   // byte offsets
  int64_t step;
};

namespace tpp {

namespace {

constexpr int kHidden = 512;

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct MlpLayout {
  int64_t woff[4], boff[4], nparams, wbf_off[4], nwbf;
  size_t p32, pbf, grad, am, av, act, pre, g0, g1, lossv, scal, total;
};

MlpLayout mlp_layout(int n, int max_batch, int32_t* widths) {
  widths[0] = 2 * n * n + 1;
  widths[1] = widths[2] = widths[3] = kHidden;
  widths[4] = 4 * n * n;
  MlpLayout L{};
  int64_t o = 0, ob = 0;
  for (int l = 0; l < 4; ++l) {
    L.woff[l] = o;
    o += (int64_t)widths[l] * widths[l + 1];
    L.boff[l] = o;
    o += widths[l + 1];
    L.wbf_off[l] = ob;
    ob += (int64_t)widths[l] * widths[l + 1];
  }
  L.nparams = o;
  L.nwbf = ob;
  int64_t actsz = 0;                // inputs of every layer and pre-activations
  for (int l = 0; l < 4; ++l) actsz += (int64_t)max_batch * widths[l];
  int64_t presz = 0;
  for (int l = 0; l < 4; ++l) presz += (int64_t)max_batch * widths[l + 1];
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t r = off;
    off = al256(off + (b ? b : 8));
    return r;
  };
  L.p32 = take(o * 4);
  L.pbf = take(ob * 2);
  L.grad = take(o * 4);
  L.am = take(o * 4);
  L.av = take(o * 4);
  L.act = take(actsz * 4);
  L.pre = take(presz * 4);
  L.g0 = take((size_t)max_batch * 4 * n * n > (size_t)max_batch * kHidden
                  ? (size_t)max_batch * 4 * n * n * 4 : (size_t)max_batch * kHidden * 4);
  L.g1 = take((size_t)max_batch * 4 * n * n > (size_t)max_batch * kHidden
                  ? (size_t)max_batch * 4 * n * n * 4 : (size_t)max_batch * kHidden * 4);
  L.lossv = take((size_t)max_batch * 8);
  L.scal = take(64);
  L.total = off;
  return L;
}

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ float gelu_f(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
         x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// C[M x N] = op(A) op(B) (+ bias[j]) (+ C if accumulate), FP32 accumulation;
// A(i, k) = A[i sai + k sak], B(k, j) = B[k sbk + j sbj].  With Cact, also
// Cact = GELU(C).  64 x 64 tiles, 256 threads, 4 x 4 outputs per thread.
template <typename TB>
__global__ void __launch_bounds__(256)
k_gemm(int M, int N, int K, const float* __restrict__ A, int64_t sai, int64_t sak,
       const TB* __restrict__ B, int64_t sbk, int64_t sbj, float* __restrict__ C, int ldc,
       const float* __restrict__ bias, float* __restrict__ Cact, int accumulate) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  float acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0f;
  const bool akfast = (sak == 1), bjfast = (sbj == 1);
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int t = threadIdx.x; t < 64 * 16; t += 256) {
      const int ii = akfast ? t / 16 : t % 64, kk = akfast ? t % 16 : t / 64;
      const int gi = i0 + ii, gk = k0 + kk;
      As[kk][ii] = (gi < M && gk < K) ? A[gi * sai + gk * sak] : 0.0f;
    }
    for (int t = threadIdx.x; t < 16 * 64; t += 256) {
      const int jj = bjfast ? t % 64 : t / 16, kk = bjfast ? t / 64 : t % 16;
      const int gj = j0 + jj, gk = k0 + kk;
      Bs[kk][jj] = (gj < N && gk < K) ? to_f(B[gk * sbk + gj * sbj]) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty * 4 + r;
    if (i >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx * 4 + c;
      if (j >= N) continue;
      float v = acc[r][c] + (bias ? bias[j] : 0.0f);
      if (accumulate) v += C[(int64_t)i * ldc + j];
      C[(int64_t)i * ldc + j] = v;
      if (Cact) Cact[(int64_t)i * ldc + j] = gelu_f(v);
    }
  }
}

template <typename TB>
void gemm(int M, int N, int K, const float* A, int64_t sai, int64_t sak, const TB* B,
          int64_t sbk, int64_t sbj, float* C, int ldc, const float* bias, float* Cact,
          int accumulate, cudaStream_t s) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  k_gemm<TB><<<grid, 256, 0, s>>>(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, bias, Cact,
                                  accumulate);
  count_launch();
}

__global__ void k_gelu_back(float* __restrict__ G, const float* __restrict__ Z, int64_t count) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    G[t] *= gelu_grad_f(Z[t]);
}

// db[j] = sum_i G[i, j] (rows in order: deterministic)
__global__ void k_colsum(const float* __restrict__ G, int rows, int cols, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float sv = 0.0f;
  for (int i = 0; i < rows; ++i) sv += G[(int64_t)i * cols + j];
  db[j] = sv;
}

__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out,
                          int64_t count) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = __float2bfloat16_rn(in[t]);
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 master weights
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t count, float lr, float c1, float c2) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float gt = g[t];
    const float mt = 0.9f * m[t] + 0.1f * gt;
    const float vt = 0.999f * v[t] + 0.001f * gt * gt;
    m[t] = mt;
    v[t] = vt;
    p[t] -= lr * (mt * c1) / (sqrtf(vt * c2) + 1e-8f);
  }
}

// off-diagonal row o of the structure basis -> vec index a + n b (a != b)
__device__ __forceinline__ int offdiag_index(int o, int n) {
  const int b = o / (n - 1), a0 = o % (n - 1), a = a0 + (a0 >= b ? 1 : 0);
  return a + n * b;
}

// Loss of one element per block and dL/d(outputs) (scaled by 1/B into dout).
// out: [B][4 nn] (float); Mn: [B][r r] (column-major core / ||M||_F); Qo [Ro][rz]
// column-major.  lossv[e] = L_e (double).
__global__ void __launch_bounds__(256)
k_factor_loss(const float* __restrict__ out, const double* __restrict__ Mn,
              const double* __restrict__ Qo, int n, int rz, int B, float inv_batch,
              float* __restrict__ dout, double* __restrict__ lossv) {
  extern __shared__ double smf[];
  const int nn = n * n, r = n + rz, Ro = nn - n;
  const int e = blockIdx.x, tid = threadIdx.x;
  double* v = smf;                  // 4 nn: a1, b1, a2, b2
  double* pj = v + 4 * nn;          // 4 r: Q^T of each
  double* mp = pj + 4 * r;          // 4 r: Mn beta_1, Mn^T alpha_1, Mn beta_2, Mn^T alpha_2
  double* red = mp + 4 * r;         // 32
  const float* oe = out + (int64_t)e * 4 * nn;
  const double* M = Mn + (int64_t)e * r * r;
  for (int q = tid; q < 4 * nn; q += blockDim.x) v[q] = (double)oe[q];
  __syncthreads();
  for (int q = tid; q < 4 * r; q += blockDim.x) {
    const int k = q / r, t = q % r;
    const double* x = v + k * nn;
    double sv = 0.0;
    if (t < n) {
      sv = x[t + n * t];
    } else {
      const double* qc = Qo + (int64_t)(t - n) * Ro;
      for (int o = 0; o < Ro; ++o) sv += qc[o] * x[offdiag_index(o, n)];
    }
    pj[q] = sv;
  }
  __syncthreads();
  // k = 0: Mn beta_1; 1: Mn^T alpha_1; 2: Mn beta_2; 3: Mn^T alpha_2
  for (int q = tid; q < 4 * r; q += blockDim.x) {
    const int k = q / r, t = q % r;
    double sv = 0.0;
    if (k == 0 || k == 2) {
      const double* beta = pj + (k + 1) * r;
      for (int c = 0; c < r; ++c) sv += M[t + (int64_t)r * c] * beta[c];
    } else {
      const double* alpha = pj + (k - 1) * r;
      for (int c = 0; c < r; ++c) sv += M[c + (int64_t)r * t] * alpha[c];
    }
    mp[q] = sv;
  }
  __syncthreads();
  // scalars: s0 = a1.a1, s1 = a1.a2, s2 = a2.a2, s3 = b1.b1, s4 = b1.b2, s5 = b2.b2,
  // s6 = alpha_1^T Mn beta_1, s7 = alpha_2^T Mn beta_2
  __shared__ double sc[8];
  if (tid < 32 * 8) {
    const int w = tid >> 5, lane = tid & 31;
    const double *x, *y;
    int len = nn;
    switch (w) {
      case 0: x = v; y = v; break;
      case 1: x = v; y = v + 2 * nn; break;
      case 2: x = v + 2 * nn; y = v + 2 * nn; break;
      case 3: x = v + nn; y = v + nn; break;
      case 4: x = v + nn; y = v + 3 * nn; break;
      case 5: x = v + 3 * nn; y = v + 3 * nn; break;
      case 6: x = pj; y = mp; len = r; break;              // alpha_1 . (Mn beta_1)
      default: x = pj + 2 * r; y = mp + 2 * r; len = r; break;
    }
    double sv = 0.0;
    for (int q = lane; q < len; q += 32) sv += x[q] * y[q];
    sv = warp_sum(sv);
    if (lane == 0) sc[w] = sv;
  }
  __syncthreads();
  const double aa11 = sc[0], aa12 = sc[1], aa22 = sc[2], bb11 = sc[3], bb12 = sc[4], bb22 = sc[5];
  if (tid == 0) {
    lossv[e] = 1.0 - 2.0 * (sc[6] + sc[7]) + aa11 * bb11 + 2.0 * aa12 * bb12 + aa22 * bb22;
  }
  if (!dout) return;
  // gradients: da_k = -2 Q (Mn beta_k) + 2 sum_l a_l (b_l . b_k); db_k likewise
  float* de = dout + (int64_t)e * 4 * nn;
  const double g = 2.0 * inv_batch;
  for (int q = tid; q < 4 * nn; q += blockDim.x) {
    const int k = q / nn, idx = q % nn;
    const int i = idx % n, j = idx / n;
    const double* y = mp + k * r;    // Q y with y = mp_k
    double qy;
    if (i == j) {
      qy = y[i];
    } else {
      const int o = j * (n - 1) + (i > j ? i - 1 : i);
      qy = 0.0;
      for (int t = 0; t < rz; ++t) qy += Qo[(int64_t)t * Ro + o] * y[n + t];
    }
    double lin;
    switch (k) {
      case 0: lin = v[idx] * bb11 + v[2 * nn + idx] * bb12; break;            // a1
      case 1: lin = v[nn + idx] * aa11 + v[3 * nn + idx] * aa12; break;       // b1
      case 2: lin = v[idx] * bb12 + v[2 * nn + idx] * bb22; break;            // a2
      default: lin = v[nn + idx] * aa12 + v[3 * nn + idx] * aa22; break;      // b2
    }
    de[q] = (float)(g * (lin - qy));
  }
}

__global__ void k_mean(const double* __restrict__ v, int count, float* __restrict__ out) {
  double sv = 0.0;
  for (int i = threadIdx.x; i < count; i += 32) sv += v[i];
  sv = warp_sum(sv);
  if (threadIdx.x == 0) *out = (float)(sv / count);
}

}  // namespace

// ---- helpers used by the context-side learned build (k_build.cu) -------------
int mlp_n(const tpp_mlp* net) { return net->n; }
int mlp_max_batch(const tpp_mlp* net) { return net->max_batch; }

void mlp_forward(tpp_mlp* net, const float* X, int B, float* out, cudaStream_t s) {
  const float* p32 = reinterpret_cast<const float*>(net->ws + net->p32);
  const __nv_bfloat16* wb = reinterpret_cast<const __nv_bfloat16*>(net->ws + net->pbf);
  float* act = reinterpret_cast<float*>(net->ws + net->act);
  float* pre = reinterpret_cast<float*>(net->ws + net->pre);
  const int* w = net->widths;
  // layer l input H_l (act), pre-activation Z_l (pre); H_0 = X (copied)
  int64_t ao = 0, po = 0;
  cudaMemcpyAsync(act, X, (size_t)B * w[0] * sizeof(float), cudaMemcpyDeviceToDevice, s);
  for (int l = 0; l < 4; ++l) {
    const float* H = act + ao;
    float* Z = pre + po;
    const bool last = (l == 3);
    float* Hn = last ? nullptr : act + ao + (int64_t)B * w[l];
    gemm<__nv_bfloat16>(B, w[l + 1], w[l], H, w[l], 1, wb + net->wbf_off[l], w[l + 1], 1, Z,
                        w[l + 1], p32 + net->boff[l], Hn, 0, s);
    ao += (int64_t)B * w[l];
    po += (int64_t)B * w[l + 1];
  }
  cudaMemcpyAsync(out, pre + po - (int64_t)B * w[4], (size_t)B * w[4] * sizeof(float),
                  cudaMemcpyDeviceToDevice, s);
}

cudaError_t mlp_factor_loss(const float* out, const double* Mn, const double* Qo, int n, int rz,
                            int B, float inv_batch, float* dout, double* lossv, cudaStream_t s) {
  const int nn = n * n, r = n + rz;
  const size_t smem = (size_t)(4 * nn + 8 * r + 32) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_factor_loss, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_factor_loss<<<B, 256, smem, s>>>(out, Mn, Qo, n, rz, B, inv_batch, dout, lossv);
  count_launch();
  return cudaGetLastError();
}

}  // namespace tpp

using namespace tpp;

extern "C" {

int64_t tpp_mlp_num_params(int32_t n) {
  if (n < 1 || n > TPP_MAX_N) return -1;
  int32_t w[5];
  return mlp_layout(n, 1, w).nparams;
}

size_t tpp_mlp_workspace_bytes(int32_t n, int32_t max_batch) {
  if (n < 2 || n > TPP_MAX_N || max_batch < 1) return 0;
  int32_t w[5];
  return mlp_layout(n, max_batch, w).total;
}

tpp_status tpp_mlp_create(tpp_mlp** out, int32_t n, int32_t max_batch, void* workspace,
                          size_t ws_bytes, void* stream) {
  if (!out) {
    set_error("out is NULL");
    return TPP_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (n < 2 || n > TPP_MAX_N || max_batch < 1) {
    set_error("n must be in [2, 32] and max_batch >= 1");
    return TPP_ERR_INVALID_ARG;
  }
  tpp_mlp* m = new tpp_mlp();
  const MlpLayout L = mlp_layout(n, max_batch, m->widths);
  if (!workspace || ws_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255u)) {
    delete m;
    set_error("workspace NULL, smaller than tpp_mlp_workspace_bytes() or not 256-byte aligned");
    return TPP_ERR_WORKSPACE;
  }
  m->n = n;
  m->max_batch = max_batch;
  for (int l = 0; l < 4; ++l) {
    m->woff[l] = L.woff[l];
    m->boff[l] = L.boff[l];
    m->wbf_off[l] = L.wbf_off[l];
  }
  m->nparams = L.nparams;
  m->ws = static_cast<char*>(workspace);
  m->ws_bytes = ws_bytes;
  m->p32 = L.p32;
  m->pbf = L.pbf;
  m->grad = L.grad;
  m->am = L.am;
  m->av = L.av;
  m->act = L.act;
  m->pre = L.pre;
  m->g0 = L.g0;
  m->g1 = L.g1;
  m->lossv = L.lossv;
  m->scal = L.scal;
  m->step = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(m->ws, 0, L.total, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete m;
    return cuda_check(e, "tpp_mlp_create");
  }
  *out = m;
  return TPP_OK;
}

void tpp_mlp_destroy(tpp_mlp* m) { delete m; }

// host params: for l = 0..3, W_l [K_l][N_l] row-major then b_l [N_l] (FP32)
tpp_status tpp_mlp_set_params(tpp_mlp* m, const float* host, void* stream) {
  if (!m || !host) {
    set_error("net and params must be non-NULL");
    return TPP_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* p32 = reinterpret_cast<float*>(m->ws + m->p32);
  cudaError_t e = cudaMemcpyAsync(p32, host, (size_t)m->nparams * 4, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_check(e, "tpp_mlp_set_params");
  __nv_bfloat16* wb = reinterpret_cast<__nv_bfloat16*>(m->ws + m->pbf);
  for (int l = 0; l < 4; ++l) {
    k_to_bf16<<<152, 256, 0, s>>>(p32 + m->woff[l], wb + m->wbf_off[l],
                                   (int64_t)m->widths[l] * m->widths[l + 1]);
    count_launch();
  }
  // fresh optimiser state
  cudaMemsetAsync(m->ws + m->am, 0, (size_t)m->nparams * 4, s);
  cudaMemsetAsync(m->ws + m->av, 0, (size_t)m->nparams * 4, s);
  m->step = 0;
  return cuda_check(cudaGetLastError(), "tpp_mlp_set_params");
}

tpp_status tpp_mlp_get_params(const tpp_mlp* m, float* host, void* stream) {
  if (!m || !host) {
    set_error("net and params must be non-NULL");
    return TPP_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(host, m->ws + m->p32, (size_t)m->nparams * 4,
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_check(e, "tpp_mlp_get_params");
}

tpp_status tpp_mlp_forward(tpp_mlp* m, const float* X, int32_t B, float* out, void* stream) {
  if (!m || !X || !out || B < 1 || B > m->max_batch) {
    set_error("tpp_mlp_forward: NULL pointer or batch outside [1, max_batch]");
    return TPP_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mlp_forward(m, X, B, out, s);
  return cuda_check(cudaGetLastError(), "tpp_mlp_forward");
}

// forward, loss and gradients (into the net's gradient buffer); with lr > 0 also
// one Adam step.  Mn: [B][r r] normalised cores; basis: a context of the same n
// (its structure basis Qo).  loss: device float, the batch mean.
tpp_status tpp_mlp_train_step(tpp_mlp* m, const tpp_ctx* basis, const float* X, const double* Mn,
                              int32_t B, float lr, float* loss, void* stream) {
  if (!m || !basis || !X || !Mn || B < 1 || B > m->max_batch || basis->n != m->n ||
      basis->dim != 2) {
    set_error("tpp_mlp_train_step: bad arguments (2D context of the same n, 1 <= B <= max)");
    return TPP_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int* w = m->widths;
  float* p32 = reinterpret_cast<float*>(m->ws + m->p32);
  __nv_bfloat16* wb = reinterpret_cast<__nv_bfloat16*>(m->ws + m->pbf);
  float* grad = reinterpret_cast<float*>(m->ws + m->grad);
  float* act = reinterpret_cast<float*>(m->ws + m->act);
  float* pre = reinterpret_cast<float*>(m->ws + m->pre);
  float* G0 = reinterpret_cast<float*>(m->ws + m->g0);
  float* G1 = reinterpret_cast<float*>(m->ws + m->g1);
  double* lossv = reinterpret_cast<double*>(m->ws + m->lossv);
  // forward (activations kept)
  int64_t aoff[4], poff[4], ao = 0, po = 0;
  cudaMemcpyAsync(act, X, (size_t)B * w[0] * sizeof(float), cudaMemcpyDeviceToDevice, s);
  for (int l = 0; l < 4; ++l) {
    aoff[l] = ao;
    poff[l] = po;
    const bool last = (l == 3);
    gemm<__nv_bfloat16>(B, w[l + 1], w[l], act + ao, w[l], 1, wb + m->wbf_off[l], w[l + 1], 1,
                        pre + po, w[l + 1], p32 + m->boff[l],
                        last ? nullptr : act + ao + (int64_t)B * w[l], 0, s);
    ao += (int64_t)B * w[l];
    po += (int64_t)B * w[l + 1];
  }
  // loss and dL/d(outputs) into G0
  cudaError_t e = mlp_factor_loss(pre + poff[3], Mn, basis->p<double>(basis->L.qo), m->n,
                                  basis->rz, B, 1.0f / B, G0, lossv, s);
  if (e != cudaSuccess) return cuda_check(e, "k_factor_loss");
  k_mean<<<1, 32, 0, s>>>(lossv, B, loss);
  count_launch();
  // backward
  float* Gc = G0;
  float* Gn = G1;
  for (int l = 3; l >= 0; --l) {
    const int K = w[l], N = w[l + 1];
    if (l < 3) {
      k_gelu_back<<<152 * 4, 256, 0, s>>>(Gc, pre + poff[l], (int64_t)B * N);
      count_launch();
    }
    // dW = H^T G  (K x N), db = column sums of G
    gemm<float>(K, N, B, act + aoff[l], 1, K, Gc, N, 1, grad + m->woff[l], N, nullptr, nullptr, 0,
                s);
    k_colsum<<<(N + 255) / 256, 256, 0, s>>>(Gc, B, N, grad + m->boff[l]);
    count_launch();
    if (l > 0) {   // dH = G W^T  (B x K)
      gemm<__nv_bfloat16>(B, K, N, Gc, N, 1, wb + m->wbf_off[l], 1, N, Gn, K, nullptr, nullptr,
                          0, s);
      float* t = Gc;
      Gc = Gn;
      Gn = t;
    }
  }
  if (lr > 0.0f) {
    m->step += 1;
    const double t = (double)m->step;
    const float c1 = (float)(1.0 / (1.0 - pow(0.9, t))), c2 = (float)(1.0 / (1.0 - pow(0.999, t)));
    k_adam<<<152 * 4, 256, 0, s>>>(p32, grad, reinterpret_cast<float*>(m->ws + m->am),
                                   reinterpret_cast<float*>(m->ws + m->av), m->nparams, lr, c1, c2);
    count_launch();
    for (int l = 0; l < 4; ++l) {
      k_to_bf16<<<152, 256, 0, s>>>(p32 + m->woff[l], wb + m->wbf_off[l], (int64_t)w[l] * w[l + 1]);
      count_launch();
    }
  }
  return cuda_check(cudaGetLastError(), "tpp_mlp_train_step");
}

tpp_status tpp_mlp_element_loss(tpp_mlp* m, const tpp_ctx* basis, const float* X,
                                const double* Mn, int32_t B, double* loss, void* stream) {
  if (!m || !basis || !X || !Mn || !loss || B < 1 || B > m->max_batch || basis->n != m->n ||
      basis->dim != 2) {
    set_error("tpp_mlp_element_loss: bad arguments (2D context of the same n, 1 <= B <= max)");
    return TPP_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* out = reinterpret_cast<float*>(m->ws + m->g0);
  mlp_forward(m, X, B, out, s);
  cudaError_t e = mlp_factor_loss(out, Mn, basis->p<double>(basis->L.qo), m->n, basis->rz, B,
                                  1.0f, nullptr, loss, s);
  if (e != cudaSuccess) return cuda_check(e, "k_factor_loss");
  return cuda_check(cudaGetLastError(), "tpp_mlp_element_loss");
}

// device pointer of the gradient buffer (same layout as the parameters)
const float* tpp_mlp_gradients(const tpp_mlp* m) {
  return m ? reinterpret_cast<const float*>(m->ws + m->grad) : nullptr;
}

}  // extern "C"
