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
//
// Every layer product runs on the tensor cores (k_tc_gemm.cu): BF16 weights times
// activations and gradients carried as BF16 pairs hi + lo (FP32 to 2^-17), FP32
// accumulation.  Per layer l (W_l [K_l][N_l], batch B):
//   forward   Z_l = H_l W_l + b_l            A = (H_l hi, lo) [B][K_l],  B = W_l^T
//             H_{l+1} = GELU(Z_l)            (fused epilogue, pair written for layer l + 1)
//   backward  dW_l = H_l^T G_l               A = H_l^T pair [K_l][B], B = G_l^T pair [N_l][B]
//             G_{l-1} = (G_l W_l^T) GELU'(Z_{l-1})   A = (G_l hi, lo), B = W_l [K_l][N_l]
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>

#include "tpp_internal.cuh"
#include "tpp_tc.cuh"

struct tpp_mlp {
  int32_t n, max_batch;
  int32_t widths[5];
  int32_t kp[4], np[4];                 // layer input / output widths padded to 64
  int32_t bp;                           // max_batch padded to 64 (transposed buffers)
  int64_t woff[4], boff[4], nparams;    // offsets (floats) of W_l [K][N] row-major and b_l
  char* ws;
  size_t ws_bytes;
  size_t p32, grad, am, av, pre, g[2], err, lossv, scal;   // byte offsets
  size_t wt[4], wk[4];                  // BF16 weights: W_l^T [N][kp], W_l [K][np]
  size_t hhi[4], hlo[4];                // layer inputs as pairs [max_batch][kp]
  size_t thi[4], tlo[4];                // transposed layer inputs [K_l][bp]
  size_t ghi[2], glo[2];                // gradients of the pre-activations as pairs
  size_t gthi, gtlo;                    // transposed gradient pair [N_l][bp]
  int64_t poff[4];                      // offsets (floats) of Z_l in pre
  int64_t step;
  // tensor maps of every operand (buffers fixed at creation, sized for max_batch)
  CUtensorMap fa[4][2], fb[4], da[4][2], db[4], wa[4][2], wb[4][2];
};

namespace tpp {

namespace {

constexpr int kHidden = 512;

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct MlpLayout {
  int64_t woff[4], boff[4], nparams, poff[4];
  int32_t kp[4], np[4], bp;
  size_t p32, grad, am, av, pre, g[2], err, lossv, scal;
  size_t wt[4], wk[4], hhi[4], hlo[4], thi[4], tlo[4], ghi[2], glo[2], gthi, gtlo;
  size_t total;
};

MlpLayout mlp_layout(int n, int max_batch, int32_t* widths) {
  widths[0] = 2 * n * n + 1;
  widths[1] = widths[2] = widths[3] = kHidden;
  widths[4] = 4 * n * n;
  MlpLayout L{};
  int64_t o = 0;
  for (int l = 0; l < 4; ++l) {
    L.woff[l] = o;
    o += (int64_t)widths[l] * widths[l + 1];
    L.boff[l] = o;
    o += widths[l + 1];
    L.kp[l] = tc::round_up(widths[l], 64);
    L.np[l] = tc::round_up(widths[l + 1], 64);
  }
  L.nparams = o;
  L.bp = tc::round_up(max_batch, 64);
  int64_t presz = 0;
  for (int l = 0; l < 4; ++l) {
    L.poff[l] = presz;
    presz += (int64_t)max_batch * widths[l + 1];
  }
  int wmax = 0, npmax = 0;
  for (int l = 0; l < 5; ++l) wmax = widths[l] > wmax ? widths[l] : wmax;
  for (int l = 0; l < 4; ++l) npmax = L.np[l] > npmax ? L.np[l] : npmax;
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t r = off;
    off = al256(off + (b ? b : 8));
    return r;
  };
  const size_t B = (size_t)max_batch;
  L.p32 = take(o * 4);
  L.grad = take(o * 4);
  L.am = take(o * 4);
  L.av = take(o * 4);
  L.pre = take(presz * 4);
  L.g[0] = take(B * wmax * 4);
  L.g[1] = take(B * wmax * 4);
  for (int l = 0; l < 4; ++l) {
    L.wt[l] = take((size_t)widths[l + 1] * L.kp[l] * 2);
    L.wk[l] = take((size_t)widths[l] * L.np[l] * 2);
    L.hhi[l] = take(B * L.kp[l] * 2);
    L.hlo[l] = take(B * L.kp[l] * 2);
    L.thi[l] = take((size_t)widths[l] * L.bp * 2);
    L.tlo[l] = take((size_t)widths[l] * L.bp * 2);
  }
  for (int q = 0; q < 2; ++q) {
    L.ghi[q] = take(B * npmax * 2);
    L.glo[q] = take(B * npmax * 2);
  }
  L.gthi = take((size_t)wmax * L.bp * 2);
  L.gtlo = take((size_t)wmax * L.bp * 2);
  L.err = take(64);
  L.lossv = take(B * 8);
  L.scal = take(64);
  L.total = off;
  return L;
}

template <typename T> T* at(const tpp_mlp* m, size_t off) {
  return reinterpret_cast<T*>(m->ws + off);
}

// tensor maps of every operand buffer of the network
cudaError_t make_maps(tpp_mlp* m) {
  const int* w = m->widths;
  const int B = m->max_batch, bp = m->bp;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
    const int kp = m->kp[l], np = m->np[l];
    const int q = (3 - l) & 1;                       // pair buffer holding G_l
    e = tc::make_map(&m->fa[l][0], m->ws + m->hhi[l], kp, B, kp);
    if (e == cudaSuccess) e = tc::make_map(&m->fa[l][1], m->ws + m->hlo[l], kp, B, kp);
    if (e == cudaSuccess) e = tc::make_map(&m->fb[l], m->ws + m->wt[l], kp, w[l + 1], kp);
    if (e == cudaSuccess) e = tc::make_map(&m->da[l][0], m->ws + m->ghi[q], np, B, np);
    if (e == cudaSuccess) e = tc::make_map(&m->da[l][1], m->ws + m->glo[q], np, B, np);
    if (e == cudaSuccess) e = tc::make_map(&m->db[l], m->ws + m->wk[l], np, w[l], np);
    if (e == cudaSuccess) e = tc::make_map(&m->wa[l][0], m->ws + m->thi[l], bp, w[l], bp);
    if (e == cudaSuccess) e = tc::make_map(&m->wa[l][1], m->ws + m->tlo[l], bp, w[l], bp);
    if (e == cudaSuccess) e = tc::make_map(&m->wb[l][0], m->ws + m->gthi, bp, w[l + 1], bp);
    if (e == cudaSuccess) e = tc::make_map(&m->wb[l][1], m->ws + m->gtlo, bp, w[l + 1], bp);
  }
  return e;
}

cudaError_t refresh_weights(tpp_mlp* m, cudaStream_t s) {
  const float* p32 = at<float>(m, m->p32);
  for (int l = 0; l < 4; ++l) {
    cudaError_t e = tc::weights_bf16(p32 + m->woff[l], m->widths[l], m->widths[l + 1],
                                     at<__nv_bfloat16>(m, m->wt[l]), m->kp[l],
                                     at<__nv_bfloat16>(m, m->wk[l]), m->np[l], s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// db[j] = sum_i G[i, j] (rows in order: deterministic)
__global__ void k_colsum(const float* __restrict__ G, int rows, int cols, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float sv = 0.0f;
  for (int i = 0; i < rows; ++i) sv += G[(int64_t)i * cols + j];
  db[j] = sv;
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


// Forward pass of B rows.  train: keep the transposed input pairs of every layer
// (for the weight gradients) and write the outputs to Z_3; otherwise to out.
cudaError_t forward_tc(tpp_mlp* m, const float* X, int B, float* out, bool train,
                       cudaStream_t s) {
  const int* w = m->widths;
  const int Mt = tc::round_up(B, 64);
  float* pre = at<float>(m, m->pre);
  const float* p32 = at<float>(m, m->p32);
  int* err = at<int>(m, m->err);
  cudaError_t e = tc::split(X, B, w[0], w[0], at<__nv_bfloat16>(m, m->hhi[0]),
                            at<__nv_bfloat16>(m, m->hlo[0]), m->kp[0],
                            train ? at<__nv_bfloat16>(m, m->thi[0]) : nullptr,
                            train ? at<__nv_bfloat16>(m, m->tlo[0]) : nullptr, m->bp, Mt, s);
  for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
    tc::Operands op;
    op.a[0] = m->fa[l][0];
    op.a[1] = m->fa[l][1];
    op.b[0] = m->fb[l];
    op.b[1] = m->fb[l];
    op.ktiles[0] = op.ktiles[1] = m->kp[l] / 64;
    op.nseg = 2;
    tc::Epilogue ep{};
    ep.M = B;
    ep.N = w[l + 1];
    ep.Mt = Mt;
    ep.bias = p32 + m->boff[l];
    ep.err = err;
    if (l < 3) {
      ep.kind = tc::kEpiHidden;
      ep.outf = train ? pre + m->poff[l] : nullptr;   // pre-activations: back-propagation only
      ep.ldo = w[l + 1];
      ep.hi = at<__nv_bfloat16>(m, m->hhi[l + 1]);
      ep.lo = at<__nv_bfloat16>(m, m->hlo[l + 1]);
      ep.ldh = m->kp[l + 1];
      if (train) {
        ep.thi = at<__nv_bfloat16>(m, m->thi[l + 1]);
        ep.tlo = at<__nv_bfloat16>(m, m->tlo[l + 1]);
        ep.ldt = m->bp;
      }
    } else {
      ep.kind = tc::kEpiF32;
      ep.outf = train ? pre + m->poff[3] : out;
      ep.ldo = w[4];
    }
    e = tc::gemm(op, ep, B, w[l + 1], s);
  }
  return e;
}

}  // namespace

// ---- helpers used by the context-side learned build (k_build.cu) -------------
int mlp_n(const tpp_mlp* net) { return net->n; }
int mlp_max_batch(const tpp_mlp* net) { return net->max_batch; }

void mlp_forward(tpp_mlp* net, const float* X, int B, float* out, cudaStream_t s) {
  forward_tc(net, X, B, out, false, s);
}

int mlp_read_error(const tpp_mlp* net, cudaStream_t s) {
  int v = 0;
  if (cudaMemcpyAsync(&v, net->ws + net->err, sizeof(int), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return -1;
  return v;
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
    m->poff[l] = L.poff[l];
    m->kp[l] = L.kp[l];
    m->np[l] = L.np[l];
    m->wt[l] = L.wt[l];
    m->wk[l] = L.wk[l];
    m->hhi[l] = L.hhi[l];
    m->hlo[l] = L.hlo[l];
    m->thi[l] = L.thi[l];
    m->tlo[l] = L.tlo[l];
  }
  m->bp = L.bp;
  m->nparams = L.nparams;
  m->ws = static_cast<char*>(workspace);
  m->ws_bytes = ws_bytes;
  m->p32 = L.p32;
  m->grad = L.grad;
  m->am = L.am;
  m->av = L.av;
  m->pre = L.pre;
  for (int q = 0; q < 2; ++q) {
    m->g[q] = L.g[q];
    m->ghi[q] = L.ghi[q];
    m->glo[q] = L.glo[q];
  }
  m->gthi = L.gthi;
  m->gtlo = L.gtlo;
  m->err = L.err;
  m->lossv = L.lossv;
  m->scal = L.scal;
  m->step = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = make_maps(m);
  if (e != cudaSuccess) {
    delete m;
    return cuda_check(e, "tpp_mlp_create: tensor maps");
  }
  e = cudaMemsetAsync(m->ws, 0, L.total, s);
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
  float* p32 = at<float>(m, m->p32);
  cudaError_t e = cudaMemcpyAsync(p32, host, (size_t)m->nparams * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = refresh_weights(m, s);
  // fresh optimiser state
  if (e == cudaSuccess) e = cudaMemsetAsync(m->ws + m->am, 0, (size_t)m->nparams * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->ws + m->av, 0, (size_t)m->nparams * 4, s);
  m->step = 0;
  return cuda_check(e, "tpp_mlp_set_params");
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
  if (e != cudaSuccess) return cuda_check(e, "tpp_mlp_get_params");
  if (mlp_read_error(m, s) != 0) {
    set_error("a tensor-core GEMM of the network gave up waiting on its pipeline");
    return TPP_ERR_TIMEOUT;
  }
  return TPP_OK;
}

tpp_status tpp_mlp_forward(tpp_mlp* m, const float* X, int32_t B, float* out, void* stream) {
  if (!m || !X || !out || B < 1 || B > m->max_batch) {
    set_error("tpp_mlp_forward: NULL pointer or batch outside [1, max_batch]");
    return TPP_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return cuda_check(forward_tc(m, X, B, out, false, s), "tpp_mlp_forward");
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
  const int Mt = tc::round_up(B, 64);
  float* p32 = at<float>(m, m->p32);
  float* grad = at<float>(m, m->grad);
  float* pre = at<float>(m, m->pre);
  double* lossv = at<double>(m, m->lossv);
  int* err = at<int>(m, m->err);
  cudaError_t e = forward_tc(m, X, B, nullptr, true, s);
  if (e != cudaSuccess) return cuda_check(e, "network forward");
  // loss and dL/d(outputs) = G_3 (FP32) into g[0], then its BF16 pair
  e = mlp_factor_loss(pre + m->poff[3], Mn, basis->p<double>(basis->L.qo), m->n, basis->rz, B,
                      1.0f / B, at<float>(m, m->g[0]), lossv, s);
  if (e != cudaSuccess) return cuda_check(e, "k_factor_loss");
  k_mean<<<1, 32, 0, s>>>(lossv, B, loss);
  count_launch();
  e = tc::split(at<float>(m, m->g[0]), B, w[4], w[4], at<__nv_bfloat16>(m, m->ghi[0]),
                at<__nv_bfloat16>(m, m->glo[0]), m->np[3], at<__nv_bfloat16>(m, m->gthi),
                at<__nv_bfloat16>(m, m->gtlo), m->bp, Mt, s);
  for (int l = 3; l >= 0 && e == cudaSuccess; --l) {
    const int q = (3 - l) & 1;
    // dW_l = H_l^T G_l: pairs (hi hi + hi lo + lo hi) over the batch
    tc::Operands op;
    op.a[0] = m->wa[l][0];
    op.a[1] = m->wa[l][0];
    op.a[2] = m->wa[l][1];
    op.b[0] = m->wb[l][0];
    op.b[1] = m->wb[l][1];
    op.b[2] = m->wb[l][0];
    op.ktiles[0] = op.ktiles[1] = op.ktiles[2] = Mt / 64;
    op.nseg = 3;
    tc::Epilogue ep{};
    ep.kind = tc::kEpiF32;
    ep.M = w[l];
    ep.N = w[l + 1];
    ep.outf = grad + m->woff[l];
    ep.ldo = w[l + 1];
    ep.err = err;
    e = tc::gemm(op, ep, w[l], w[l + 1], s);
    if (e != cudaSuccess) break;
    // db_l = column sums of G_l
    k_colsum<<<(w[l + 1] + 255) / 256, 256, 0, s>>>(at<float>(m, m->g[q]), B, w[l + 1],
                                                     grad + m->boff[l]);
    count_launch();
    if (l == 0) break;
    // G_{l-1} = (G_l W_l^T) GELU'(Z_{l-1})
    tc::Operands od;
    od.a[0] = m->da[l][0];
    od.a[1] = m->da[l][1];
    od.b[0] = m->db[l];
    od.b[1] = m->db[l];
    od.ktiles[0] = od.ktiles[1] = m->np[l] / 64;
    od.nseg = 2;
    tc::Epilogue eg{};
    eg.kind = tc::kEpiGeluBack;
    eg.M = B;
    eg.N = w[l];
    eg.Mt = Mt;
    eg.zprev = pre + m->poff[l - 1];
    eg.ldz = w[l];
    eg.outf = at<float>(m, m->g[1 - q]);
    eg.ldo = w[l];
    eg.hi = at<__nv_bfloat16>(m, m->ghi[1 - q]);
    eg.lo = at<__nv_bfloat16>(m, m->glo[1 - q]);
    eg.ldh = m->np[l - 1];
    eg.thi = at<__nv_bfloat16>(m, m->gthi);
    eg.tlo = at<__nv_bfloat16>(m, m->gtlo);
    eg.ldt = m->bp;
    eg.err = err;
    e = tc::gemm(od, eg, B, w[l], s);
  }
  if (e != cudaSuccess) return cuda_check(e, "network backward");
  if (lr > 0.0f) {
    m->step += 1;
    const double t = (double)m->step;
    const float c1 = (float)(1.0 / (1.0 - pow(0.9, t))), c2 = (float)(1.0 / (1.0 - pow(0.999, t)));
    k_adam<<<152 * 4, 256, 0, s>>>(p32, grad, at<float>(m, m->am), at<float>(m, m->av),
                                   m->nparams, lr, c1, c2);
    count_launch();
    e = refresh_weights(m, s);
    if (e != cudaSuccess) return cuda_check(e, "BF16 weights");
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
  float* out = at<float>(m, m->g[0]);
  cudaError_t e = forward_tc(m, X, B, out, false, s);
  if (e != cudaSuccess) return cuda_check(e, "network forward");
  e = mlp_factor_loss(out, Mn, basis->p<double>(basis->L.qo), m->n, basis->rz, B, 1.0f, nullptr,
                      loss, s);
  if (e != cudaSuccess) return cuda_check(e, "k_factor_loss");
  return cuda_check(cudaGetLastError(), "tpp_mlp_element_loss");
}

// device pointer of the gradient buffer (same layout as the parameters)
const float* tpp_mlp_gradients(const tpp_mlp* m) {
  return m ? reinterpret_cast<const float*>(m->ws + m->grad) : nullptr;
}

}  // extern "C"
