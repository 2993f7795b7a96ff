// Kronecker preconditioner apply in BF16 on the tensor cores (2D, n <= 16, the
// one-sided form of Alg. 2d-apply): for every right-hand side B of an element,
//   R = L_B^-1 (B S_A^T),   C2 Z + Z T1^T = R by columns from the last with the
//   stored shifted inverses (z_j = Gs_j r^_j + Gp_j r^_p),   X = Z Q1^T.
// With several right-hand sides per element every stage is a dense contraction:
// one CTA per element, each warp carries 8 right-hand sides, and every product
// runs as mma.sync.m16n8k16 (BF16 operands, FP32 accumulation): stage inputs and
// factors are rounded to BF16, sums are FP32.  Matrices are padded to 16 x 16 with
// zeros.  The per-element blocks (16 x 16 x 16 products, 16 x 8 sweep tiles) are
// below the smallest tcgen05 tile (M = 64), hence the warp-level instruction.
#include <cuda_bf16.h>

#include "tpp_internal.cuh"

namespace tpp {

namespace {

constexpr int kT = 16;          // padded order
constexpr int kRT = 8;          // right-hand sides per warp tile
constexpr int kWarps = 4;
constexpr int kPad = kT + 1;    // row stride of the per-warp fp32 buffers

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x (low half) = lo
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t ld2(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

// d += A B for one m16n8k16 tile (BF16 A row-major 16 x 16, B 16 x 8, FP32 d)
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A fragment of a row-major 16 x 16 BF16 matrix in shared memory
__device__ __forceinline__ void frag_a(const __nv_bfloat16* M, int g, int c, uint32_t* a) {
  a[0] = ld2(M + g * kT + 2 * c);
  a[1] = ld2(M + (g + 8) * kT + 2 * c);
  a[2] = ld2(M + g * kT + 2 * c + 8);
  a[3] = ld2(M + (g + 8) * kT + 2 * c + 8);
}

struct TcFactors {      // BF16 copies (row-major, per element), see k_bf16_factors
  const __nv_bfloat16 *SA, *LB, *Q1, *G;
  const float* T1u;
  const uint32_t* masks;
};

template <typename VT>
__global__ void __launch_bounds__(kWarps * 32)
k_apply_2d_tc(int n, int R, TcFactors F, const VT* __restrict__ b, VT* __restrict__ x,
              const int32_t* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  __nv_bfloat16* SA = reinterpret_cast<__nv_bfloat16*>(smraw);
  __nv_bfloat16* LB = SA + kT * kT;
  __nv_bfloat16* Q1 = LB + kT * kT;
  __nv_bfloat16* G = Q1 + kT * kT;                       // [16][2][16 x 16]
  float* T1u = reinterpret_cast<float*>(G + kT * 2 * kT * kT);
  float* wbuf = T1u + kT * kT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, c = lane & 3;
  float(*RT)[kT][kPad] = reinterpret_cast<float(*)[kT][kPad]>(wbuf + warp * 2 * kRT * kT * kPad);
  float(*ZT)[kT][kPad] = RT + kRT;
  const int64_t e = blockIdx.x;
  const int nn = n * n;
  // ---- factors of the element, zero-padded to 16 x 16
  for (int q = threadIdx.x; q < kT * kT; q += blockDim.x) {
    const int r = q / kT, cc = q % kT;
    const bool ok = r < n && cc < n;
    const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
    SA[q] = ok ? F.SA[e * nn + r * n + cc] : z;
    LB[q] = ok ? F.LB[e * nn + r * n + cc] : z;
    Q1[q] = ok ? F.Q1[e * nn + r * n + cc] : z;
    T1u[q] = ok ? F.T1u[e * nn + r * n + cc] : 0.0f;
  }
  for (int q = threadIdx.x; q < kT * 2 * kT * kT; q += blockDim.x) {
    const int j = q / (2 * kT * kT), s = (q / (kT * kT)) % 2, rc = q % (kT * kT);
    const int r = rc / kT, cc = rc % kT;
    G[q] = (j < n && r < n && cc < n) ? F.G[(e * n + j) * 2 * nn + s * nn + r * n + cc]
                                      : __float2bfloat16_rn(0.0f);
  }
  __syncthreads();
  // 2x2 blocks of T1: cst bit r = a block starts at column r
  uint32_t cst = 0;
  {
    const uint32_t m1 = F.masks[2 * e];
    int r = 0;
    while (r < n) {
      const bool two = ((m1 >> r) & 1u) && r + 1 < n;
      if (two) cst |= 1u << r;
      r += two ? 2 : 1;
    }
  }
  uint32_t asa[4];
  const int ntiles = (R + kRT - 1) / kRT;
  for (int tile = warp; tile < ntiles; tile += kWarps) {
    for (int q = lane; q < kRT * kT * kPad; q += 32) (&ZT[0][0][0])[q] = 0.0f;
    // ---- stages 1-2 for each right-hand side of the tile: R^T = (S_A B^T) L_B^-T
    for (int rr = 0; rr < kRT; ++rr) {
      const int rhs = tile * kRT + rr;
      if (rhs >= R) {                                    // padding columns of the sweep
        for (int q = lane; q < kT * kPad; q += 32) (&RT[rr][0][0])[q] = 0.0f;
        continue;
      }
      const VT* bb = b + (e * R + rhs) * nn;
      frag_a(SA, g, c, asa);
      float w[2][4];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        // B operand element (k = j, n = i) = B[i][j] = b[i + n j]
        const int i = 8 * t + g;
        auto bv = [&](int j) -> float {
          return (i < n && j < n) ? (float)bb[i + n * j] : 0.0f;
        };
        w[t][0] = w[t][1] = w[t][2] = w[t][3] = 0.0f;
        mma16816(w[t], asa, pack2(bv(2 * c), bv(2 * c + 1)), pack2(bv(2 * c + 8), bv(2 * c + 9)));
      }
      // W^T (rows j, cols i) as the A operand of the next product
      const uint32_t aw[4] = {pack2(w[0][0], w[0][1]), pack2(w[0][2], w[0][3]),
                              pack2(w[1][0], w[1][1]), pack2(w[1][2], w[1][3])};
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        const int q = 8 * t + g;                           // B element (k = i, n = q) = L_B^-1[q][i]
        mma16816(d, aw, ld2(LB + q * kT + 2 * c), ld2(LB + q * kT + 2 * c + 8));
        RT[rr][g][8 * t + 2 * c] = d[0];
        RT[rr][g][8 * t + 2 * c + 1] = d[1];
        RT[rr][g + 8][8 * t + 2 * c] = d[2];
        RT[rr][g + 8][8 * t + 2 * c + 1] = d[3];
      }
    }
    __syncwarp();
    // ---- sweep over the columns of R (rows of R^T), last first, 8 right-hand sides at once
    for (int jj = n - 1; jj >= 0; --jj) {
      const bool lo = (cst >> jj) & 1u;                          // first column of a pair
      const bool up = jj >= 1 && ((cst >> (jj - 1)) & 1u);      // second column of a pair
      const int jp = up ? jj - 1 : jj + 1;                      // partner column
      float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      uint32_t ag[4];
      frag_a(G + (jj * 2 + 0) * kT * kT, g, c, ag);
      // B operand element (k = i', n = r) = r-th right-hand side's column jj, row i'
      mma16816(d, ag, pack2(RT[g][jj][2 * c], RT[g][jj][2 * c + 1]),
               pack2(RT[g][jj][2 * c + 8], RT[g][jj][2 * c + 9]));
      if (lo || up) {
        frag_a(G + (jj * 2 + 1) * kT * kT, g, c, ag);
        mma16816(d, ag, pack2(RT[g][jp][2 * c], RT[g][jp][2 * c + 1]),
                 pack2(RT[g][jp][2 * c + 8], RT[g][jp][2 * c + 9]));
      }
      // d = z(i, r) for i = g, g + 8 and r = 2c, 2c + 1
      ZT[2 * c][jj][g] = d[0];
      ZT[2 * c + 1][jj][g] = d[1];
      ZT[2 * c][jj][g + 8] = d[2];
      ZT[2 * c + 1][jj][g + 8] = d[3];
      for (int k = 0; k < jj; ++k) {        // the remaining columns (in-block entries are 0)
        const float t = T1u[k * kT + jj];
        RT[2 * c][k][g] -= t * d[0];
        RT[2 * c + 1][k][g] -= t * d[1];
        RT[2 * c][k][g + 8] -= t * d[2];
        RT[2 * c + 1][k][g + 8] -= t * d[3];
      }
      __syncwarp();
    }
    // ---- stage 4 for each right-hand side: X = Z Q1^T
    for (int rr = 0; rr < kRT; ++rr) {
      const int rhs = tile * kRT + rr;
      if (rhs >= R) break;
      // A operand element (i, j) = Z[i][j] = ZT[rr][j][i]
      const uint32_t az[4] = {pack2(ZT[rr][2 * c][g], ZT[rr][2 * c + 1][g]),
                              pack2(ZT[rr][2 * c][g + 8], ZT[rr][2 * c + 1][g + 8]),
                              pack2(ZT[rr][2 * c + 8][g], ZT[rr][2 * c + 9][g]),
                              pack2(ZT[rr][2 * c + 8][g + 8], ZT[rr][2 * c + 9][g + 8])};
      VT* xx = x + (e * R + rhs) * nn;
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        const int col = 8 * t + g;                         // B element (k = j, n = col) = Q1[col][j]
        mma16816(d, az, ld2(Q1 + col * kT + 2 * c), ld2(Q1 + col * kT + 2 * c + 8));
        const int c0 = 8 * t + 2 * c;
        if (g < n && c0 < n) xx[g + n * c0] = (VT)d[0];
        if (g < n && c0 + 1 < n) xx[g + n * (c0 + 1)] = (VT)d[1];
        if (g + 8 < n && c0 < n) xx[g + 8 + n * c0] = (VT)d[2];
        if (g + 8 < n && c0 + 1 < n) xx[g + 8 + n * (c0 + 1)] = (VT)d[3];
      }
    }
    __syncwarp();
  }
}

// BF16 row-major copies of the one-sided apply factors (rounded to nearest) and T1
// with its diagonal 1x1 / 2x2 blocks removed (float, row-major); one thread per entry
__global__ void k_bf16_factors(int n, int64_t E, const double* SA, const double* LBi,
                               const double* Q1, const double* T1, const double* G,
                               const uint32_t* masks, __nv_bfloat16* SAr, __nv_bfloat16* LBr,
                               __nv_bfloat16* Q1r, float* T1ur, __nv_bfloat16* Gr) {
  const int nn = n * n;
  const int64_t tot = E * (int64_t)nn * (4 + 2 * n);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / ((int64_t)nn * (4 + 2 * n));
    const int64_t rem = q % ((int64_t)nn * (4 + 2 * n));
    if (rem < 4 * nn) {
      const int which = (int)(rem / nn), rc = (int)(rem % nn);
      const int r = rc / n, cc = rc % n;            // row-major (r, cc); sources column-major
      const int64_t src = e * nn + r + (int64_t)n * cc;
      if (which == 0) SAr[e * nn + rc] = __double2bfloat16(SA[src]);
      else if (which == 1) LBr[e * nn + rc] = __double2bfloat16(LBi[src]);
      else if (which == 2) Q1r[e * nn + rc] = __double2bfloat16(Q1[src]);
      else {
        const uint32_t m1 = masks[2 * e];
        // block starts as the apply kernels read them
        uint32_t cst = 0;
        int k = 0;
        while (k < n) {
          const bool two = ((m1 >> k) & 1u) && k + 1 < n;
          if (two) cst |= 1u << k;
          k += two ? 2 : 1;
        }
        const bool inblk = (r == cc) || (r + 1 == cc && ((cst >> r) & 1u)) ||
                           (cc + 1 == r && ((cst >> cc) & 1u));
        T1ur[e * nn + rc] = inblk ? 0.0f : (float)T1[src];
      }
    } else {
      // G: column-major Gs_j, Gp_j ([j][s][k][i]) -> row-major [j][s][i][k]
      const int64_t gr = rem - 4 * nn;
      const int js = (int)(gr / nn), rc = (int)(gr % nn);
      const int r = rc / n, cc = rc % n;
      Gr[(e * 2 * n + js) * nn + rc] = __double2bfloat16(G[(e * 2 * n + js) * nn + r + (int64_t)n * cc]);
    }
  }
}

}  // namespace

size_t bf16_factor_bytes(int n, int64_t E) {
  const size_t nn = (size_t)n * n;
  return (size_t)E * nn * (3 * 2 + 4 + 2 * n * 2) + 4 * 256;
}

// offsets inside the BF16 region (bytes, 256-aligned pieces)
struct Bf16Layout {
  size_t SA, LB, Q1, T1u, G;
};
static Bf16Layout bf16_layout(int n, int64_t E) {
  const size_t m = (size_t)E * n * n;
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  Bf16Layout L;
  L.SA = 0;
  L.LB = al(L.SA + m * 2);
  L.Q1 = al(L.LB + m * 2);
  L.T1u = al(L.Q1 + m * 2);
  L.G = al(L.T1u + m * 4);
  return L;
}

cudaError_t launch_to_bf16(const tpp_ctx* c, cudaStream_t s) {
  const Bf16Layout B = bf16_layout(c->n, c->E);
  char* base = c->ws + c->L.bf16;
  k_bf16_factors<<<152 * 4, 256, 0, s>>>(
      c->n, c->E, c->p<double>(c->L.fSA), c->p<double>(c->L.fSB), c->p<double>(c->L.fQ1),
      c->p<double>(c->L.fT1), c->p<double>(c->L.fG), c->p<uint32_t>(c->L.masks),
      reinterpret_cast<__nv_bfloat16*>(base + B.SA), reinterpret_cast<__nv_bfloat16*>(base + B.LB),
      reinterpret_cast<__nv_bfloat16*>(base + B.Q1), reinterpret_cast<float*>(base + B.T1u),
      reinterpret_cast<__nv_bfloat16*>(base + B.G));
  count_launch();
  return cudaGetLastError();
}

template <typename VT>
cudaError_t launch_apply_bf16_t(const tpp_ctx* c, const VT* b, VT* x, const int32_t* skip,
                                cudaStream_t s) {
  const Bf16Layout B = bf16_layout(c->n, c->E);
  const char* base = c->ws + c->L.bf16;
  TcFactors F;
  F.SA = reinterpret_cast<const __nv_bfloat16*>(base + B.SA);
  F.LB = reinterpret_cast<const __nv_bfloat16*>(base + B.LB);
  F.Q1 = reinterpret_cast<const __nv_bfloat16*>(base + B.Q1);
  F.G = reinterpret_cast<const __nv_bfloat16*>(base + B.G);
  F.T1u = reinterpret_cast<const float*>(base + B.T1u);
  F.masks = c->p<uint32_t>(c->L.masks);
  const size_t smem = (size_t)kT * kT * 2 * 3 + (size_t)kT * 2 * kT * kT * 2 + kT * kT * 4 +
                      (size_t)kWarps * 2 * kRT * kT * kPad * 4;
  cudaError_t e = cudaFuncSetAttribute(k_apply_2d_tc<VT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_apply_2d_tc<VT><<<(unsigned)c->E, kWarps * 32, smem, s>>>(c->n, c->R, F, b, x, skip);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_apply_bf16(const tpp_ctx* c, const double* b, double* x, const int32_t* skip,
                              cudaStream_t s) {
  return launch_apply_bf16_t<double>(c, b, x, skip, s);
}
cudaError_t launch_apply_bf16_f32(const tpp_ctx* c, const float* b, float* x,
                                  const int32_t* skip, cudaStream_t s) {
  return launch_apply_bf16_t<float>(c, b, x, skip, s);
}

}  // namespace tpp
