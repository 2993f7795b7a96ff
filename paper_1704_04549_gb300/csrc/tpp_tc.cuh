// Tensor-core (tcgen05) GEMM of the factor network: operands, epilogues and the
// host launchers (k_tc_gemm.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tpp {
namespace tc {

// Up to three (A, B) segments summed into one FP32 accumulator.  Tensor maps of
// BF16 matrices stored K-major (rows of the contraction index), box 64 x 128,
// 128-byte swizzle (make_map); ktiles[s] = contraction length of segment s / 64.
struct Operands {
  CUtensorMap a[3];
  CUtensorMap b[3];
  int ktiles[3];
  int nseg;
};

enum { kEpiF32 = 0, kEpiHidden = 1, kEpiGeluBack = 2 };

// Epilogue of one output tile (rows m < M and columns n < N are written):
//  kEpiF32:      outf[m][n] = acc (+ bias[n])
//  kEpiHidden:   z = acc + bias[n]; outf[m][n] = z (if outf != NULL); v = GELU(z)
//  kEpiGeluBack: v = acc * GELU'(zprev[m][n]); outf[m][n] = v
// and for the last two the BF16 pair of v: hi/lo[m][n] (row stride ldh) and, when
// thi != NULL, transposed thi/tlo[n][m] (stride ldt) for every m < Mt, zero for
// m >= M.  err: set to 1 when a pipeline wait gave up (the tile is then not written).
struct Epilogue {
  int kind;
  int M, N, Mt;
  const float* bias;
  float* outf;
  int ldo;
  const float* zprev;
  int ldz;
  __nv_bfloat16* hi;
  __nv_bfloat16* lo;
  int ldh;
  __nv_bfloat16* thi;
  __nv_bfloat16* tlo;
  int ldt;
  int* err;
};

// Tensor map over a row-major BF16 matrix with `rows` rows of `row_elems`
// elements, of which the first `inner` (a multiple of 64) are read.
cudaError_t make_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t rows,
                     uint64_t row_elems);
// D[M x N] (tiles of 128 x 128) through the epilogue
cudaError_t gemm(const Operands& op, const Epilogue& ep, int M, int N, cudaStream_t s);
// BF16 pair of an FP32 matrix X [M][K] (leading dimension ldx) into hi/lo [M][ldh],
// zero-padded for K <= k < ldh, and with thi the transposed pair [K][ldt] for
// m < Mt (zero for m >= M)
cudaError_t split(const float* X, int M, int K, int ldx, __nv_bfloat16* hi, __nv_bfloat16* lo,
                  int ldh, __nv_bfloat16* thi, __nv_bfloat16* tlo, int ldt, int Mt,
                  cudaStream_t s);
// BF16 copies of W [K][N] (FP32): Wt [N][ldt] transposed (zero for K <= k < ldt)
// and Wk [K][ldk] (zero for N <= n < ldk)
cudaError_t weights_bf16(const float* W, int K, int N, __nv_bfloat16* Wt, int ldt,
                         __nv_bfloat16* Wk, int ldk, cudaStream_t s);

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

}  // namespace tc
}  // namespace tpp
