// Tensor-core GEMM of the factor network for sm_103a.
//
//   D[M x N] = sum over segments s of A_s[M x K_s] B_s[N x K_s]^T
//
// BF16 operands, both K-major, staged by TMA into shared memory with the
// 128-byte swizzle; tcgen05.mma (kind::f16, cta_group::1, M = 128, N = 128,
// K = 16 per instruction) issued by one thread, FP32 accumulators in tensor
// memory, read back by tcgen05.ld for a fused epilogue.  Persistent CTAs (one
// per SM) walk the 128 x 128 output tiles; a 4-stage mbarrier pipeline feeds the
// MMA thread, and two tensor-memory accumulators let sixteen epilogue warps drain
// one tile while the next one is multiplied.  Up to three (A, B) segments are
// summed into one accumulator; the
// network uses them to carry FP32 values as BF16 pairs v = hi + lo
// (hi = bf16(v), lo = bf16(v - hi), 16 mantissa bits): a product of an FP32
// activation with a BF16 weight is hi w + lo w, and of two FP32 operands
// hi_a hi_b + hi_a lo_b + lo_a hi_b (the lo lo term, 2^-18 relative, dropped).
//
// Every wait on an mbarrier is bounded (2 s of %globaltimer); a wait that gives
// up raises a flag that stops the other roles, the TMA thread waits (bounded)
// for its copies in flight, tensor memory is freed and the kernel writes its
// error word instead of the tile.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "tpp_internal.cuh"
#include "tpp_tc.cuh"

namespace tpp {
namespace tc {

namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64, kStages = 6;
constexpr int kABytes = kBM * kBK * 2;       // 16 KB per A tile
constexpr int kBBytes = kBN * kBK * 2;       // 16 KB per B tile
constexpr int kStageBytes = kABytes + kBBytes;
constexpr uint64_t kWaitNs = 2000000000ull;  // give up a wait after 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of parity `parity` to complete.  Gives up (returns false)
// after kWaitNs, or as soon as *abort is set when watch_abort; a wait that times
// out sets *abort so the other roles stop too.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort, bool watch_abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!mbar_try_wait(bar, parity)) {
    if (watch_abort && *abort) return false;
    if (gtimer() - t0 > kWaitNs) {
      *abort = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 64 BF16 (128 B), 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);        // start address
  d |= (uint64_t)(16u >> 4) << 16;                // leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024u >> 4) << 32;              // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                         // descriptor version (tcgen05)
  d |= (uint64_t)2 << 61;                         // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = kBN, M = kBM.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                            ((uint32_t)(kBN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float gelu_f(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
         x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// Epilogue of one 32 x 32 block of the tile (rows mb.., columns nb..), run by one
// warp straight from the tensor-memory load: lane = row mb + lane, acc[j] = column
// nb + j.  Row-major outputs leave as 16-byte vector stores of the lane's row (no
// shared-memory staging, which leaves the shared memory to the operand pipeline);
// the transposed BF16 pair (training) is written column by column with lane = row,
// coalesced over the warp.
__device__ __forceinline__ void epilogue_block(const Epilogue& ep, int mb, int nb, float* acc) {
  const int lane = threadIdx.x & 31;
  const int m = mb + lane;
  const bool row_ok = m < ep.M;
  const bool full = nb + 32 <= ep.N;                  // warp-uniform
  if (ep.kind == kEpiF32) {
    if (!row_ok) return;
    float* o = ep.outf + (int64_t)m * ep.ldo + nb;
#pragma unroll
    for (int g = 0; g < 32; g += 4) {
      float v[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int n = nb + g + t;
        v[t] = acc[g + t] + ((ep.bias && n < ep.N) ? ep.bias[n] : 0.0f);
      }
      if (full) {
        *reinterpret_cast<float4*>(o + g) = make_float4(v[0], v[1], v[2], v[3]);
      } else {
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (nb + g + t < ep.N) o[g + t] = v[t];
      }
    }
    return;
  }
  uint32_t hl[32];                                    // packed (hi, lo) of every column
#pragma unroll
  for (int g = 0; g < 32; g += 4) {
    float z[4], v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int n = nb + g + t;
      const bool ok = row_ok && n < ep.N;
      if (ep.kind == kEpiHidden) {
        z[t] = acc[g + t] + ((ep.bias && n < ep.N) ? ep.bias[n] : 0.0f);
        v[t] = ok ? gelu_f(z[t]) : 0.0f;
      } else {
        v[t] = ok ? acc[g + t] * gelu_grad_f(ep.zprev[(int64_t)m * ep.ldz + n]) : 0.0f;
        z[t] = v[t];
      }
      const __nv_bfloat16 hi = __float2bfloat16_rn(v[t]);
      const __nv_bfloat16 lo = __float2bfloat16_rn(v[t] - __bfloat162float(hi));
      hl[g + t] = (uint32_t)__bfloat16_as_ushort(hi) | ((uint32_t)__bfloat16_as_ushort(lo) << 16);
    }
    if (ep.outf && row_ok) {                          // pre-activation / gradient, FP32
      float* o = ep.outf + (int64_t)m * ep.ldo + nb + g;
      if (full) {
        *reinterpret_cast<float4*>(o) = make_float4(z[0], z[1], z[2], z[3]);
      } else {
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (nb + g + t < ep.N) o[t] = z[t];
      }
    }
  }
  if (row_ok) {                                       // the BF16 pair, row-major
    __nv_bfloat16* ph = ep.hi + (int64_t)m * ep.ldh + nb;
    __nv_bfloat16* pl = ep.lo + (int64_t)m * ep.ldh + nb;
    if (full) {
#pragma unroll
      for (int g = 0; g < 32; g += 8) {
        uint4 h4, l4;
        h4.x = (hl[g] & 0xFFFFu) | (hl[g + 1] << 16);
        h4.y = (hl[g + 2] & 0xFFFFu) | (hl[g + 3] << 16);
        h4.z = (hl[g + 4] & 0xFFFFu) | (hl[g + 5] << 16);
        h4.w = (hl[g + 6] & 0xFFFFu) | (hl[g + 7] << 16);
        l4.x = (hl[g] >> 16) | (hl[g + 1] & 0xFFFF0000u);
        l4.y = (hl[g + 2] >> 16) | (hl[g + 3] & 0xFFFF0000u);
        l4.z = (hl[g + 4] >> 16) | (hl[g + 5] & 0xFFFF0000u);
        l4.w = (hl[g + 6] >> 16) | (hl[g + 7] & 0xFFFF0000u);
        *reinterpret_cast<uint4*>(ph + g) = h4;
        *reinterpret_cast<uint4*>(pl + g) = l4;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (nb + j < ep.N) {
          ph[j] = __ushort_as_bfloat16((unsigned short)(hl[j] & 0xFFFFu));
          pl[j] = __ushort_as_bfloat16((unsigned short)(hl[j] >> 16));
        }
    }
  }
  if (ep.thi && m < ep.Mt) {                          // transposed pair (zero for m >= M)
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (nb + j < ep.N) {
        ep.thi[(int64_t)(nb + j) * ep.ldt + m] = __ushort_as_bfloat16((unsigned short)(hl[j] & 0xFFFFu));
        ep.tlo[(int64_t)(nb + j) * ep.ldt + m] = __ushort_as_bfloat16((unsigned short)(hl[j] >> 16));
      }
  }
}

// Persistent kernel: CTA c takes output tiles c, c + gridDim.x, ... (tile t is row
// block t / ntn, column block t % ntn).  Warp 0: TMA producer; warp 1: MMA issuer
// into one of two tensor-memory accumulators (columns 0..127 and 128..255), so the
// epilogue of a tile overlaps the MMAs of the next; warps 2..17: epilogue, warp w
// reading lanes 32 (w % 4) .. + 31 (the rows it may access) and columns 32 h .. + 31,
// h = (w - 2) / 4.
constexpr int kEpiWarps = 16;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kTmemCols = 2 * kBN;

__global__ void __launch_bounds__(kThreads, 1)
k_gemm_tc(const __grid_constant__ Operands op, const Epilogue ep) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], tfull[2], tempty[2], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = smem_u32(smem);
  const int ntn = (ep.N + kBN - 1) / kBN, ntm = (ep.M + kBM - 1) / kBM;
  const int ntiles = ntn * ntm;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      mbar_init(smem_u32(&tempty[b]), kEpiWarps);
    }
    mbar_init(smem_u32(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* abort = &abort_flag;

  if (warp == 0) {
    if (lane == 0) {   // TMA producer
      int it = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
        const int m0 = (t / ntn) * kBM, n0 = (t % ntn) * kBN;
        for (int sg = 0; sg < op.nseg && !*abort; ++sg) {
          for (int kt = 0; kt < op.ktiles[sg]; ++kt, ++it) {
            const int s = it % kStages;
            const uint32_t r = it / kStages;
            if (r > 0 && !mbar_wait(smem_u32(&empty[s]), (r - 1) & 1, abort, true)) break;
            const uint32_t sa = sbase + s * kStageBytes, sb = sa + kABytes;
            mbar_expect_tx(smem_u32(&full[s]), kStageBytes);
            tma_load_2d(sa, &op.a[sg], kt * kBK, m0, smem_u32(&full[s]));
            tma_load_2d(sb, &op.b[sg], kt * kBK, n0, smem_u32(&full[s]));
          }
        }
      }
      // copies in flight land before the CTA may exit (the last phase armed on each
      // stage has completed; immediate after a normal run)
      const int first = it > kStages ? it - kStages : 0;
      for (int j = first; j < it; ++j)
        mbar_wait(smem_u32(&full[j % kStages]), (j / kStages) & 1, abort, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      int it = 0, i = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x, ++i) {
        const int b = i & 1;
        const uint32_t u = i >> 1;
        if (u > 0 && !mbar_wait(smem_u32(&tempty[b]), (u - 1) & 1, abort, true)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * kBN);
        int kk = 0;
        for (int sg = 0; sg < op.nseg && !stop; ++sg) {
          for (int kt = 0; kt < op.ktiles[sg]; ++kt, ++it, ++kk) {
            const int s = it % kStages;
            const uint32_t r = it / kStages;
            if (!mbar_wait(smem_u32(&full[s]), r & 1, abort, true)) {
              stop = true;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = sbase + s * kStageBytes, sb = sa + kABytes;
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)
              mma_bf16(d, smem_desc(sa + 32 * k), smem_desc(sb + 32 * k), (kk | k) != 0);
            mma_commit(smem_u32(&empty[s]));     // frees the stage once these MMAs are done
          }
        }
        if (!stop) mma_commit(smem_u32(&tfull[b]));   // accumulator b ready
      }
      mma_commit(smem_u32(&done));      // arrives when every MMA issued above is done
    }
  } else {
    // epilogue warps
    const int e = warp - 2, q = warp & 3, h = e >> 2;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int b = i & 1;
      const uint32_t u = i >> 1;
      if (!mbar_wait(smem_u32(&tfull[b]), u & 1, abort, true)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int m0 = (t / ntn) * kBM, n0 = (t % ntn) * kBN;
      const int col = h * 32;
      if (n0 + col < ep.N) {              // warp-uniform
        float acc[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * kBN + col), acc);
        epilogue_block(ep, m0 + q * 32, n0 + col, acc);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                      smem_u32(&tempty[b]))
                                  : "memory");
    }
  }
  __syncwarp();
  // every MMA has completed before tensor memory is released
  const bool ok = mbar_wait(smem_u32(&done), 0, abort, false);
  if ((!ok || *abort) && threadIdx.x == 0) atomicExch(ep.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
cudaError_t g_encode_err = cudaSuccess;

}  // namespace

cudaError_t make_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t rows,
                     uint64_t row_elems) {
  std::call_once(g_encode_once, [] {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    g_encode_err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                    cudaEnableDefault, &q);
    if (g_encode_err == cudaSuccess && q != cudaDriverEntryPointSuccess)
      g_encode_err = cudaErrorNotSupported;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (g_encode_err != cudaSuccess) return g_encode_err;
  // inner extent a multiple of 64 elements (the box width), rows of 16-byte multiples
  if (inner % kBK != 0 || row_elems % 8 != 0 || inner > row_elems ||
      (reinterpret_cast<uintptr_t>(base) & 15u))
    return cudaErrorInvalidValue;
  const cuuint64_t dims[2] = {inner, rows};
  const cuuint64_t strides[1] = {row_elems * 2};
  const cuuint32_t box[2] = {kBK, 128};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
                              dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t gemm(const Operands& op, const Epilogue& ep, int M, int N, cudaStream_t s) {
  constexpr int kSmemBytes = kStages * kStageBytes + 1024;   // + alignment slack
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  static int num_sms = 0;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kSmemBytes);
    int dev = 0;
    if (attr_err == cudaSuccess) attr_err = cudaGetDevice(&dev);
    if (attr_err == cudaSuccess)
      attr_err = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  });
  if (attr_err != cudaSuccess) return attr_err;
  if (M < 1 || N < 1 || op.nseg < 1 || op.nseg > 3 || ep.M != M || ep.N != N)
    return cudaErrorInvalidValue;
  const int tiles = ((N + kBN - 1) / kBN) * ((M + kBM - 1) / kBM);
  const int grid = tiles < num_sms ? tiles : num_sms;
  k_gemm_tc<<<grid, kThreads, kSmemBytes, s>>>(op, ep);
  count_launch();
  return cudaGetLastError();
}

// ---- BF16 pairs of FP32 matrices -------------------------------------------

namespace {

// X [M][K] (ld ldx, FP32) -> hi/lo [M][ldh] (zero for k >= K) and, with thi,
// the transposed pair [K][ldt] for rows m < Mt (zero for m >= M).  32 x 32 tiles.
__global__ void k_split(const float* __restrict__ X, int M, int K, int ldx,
                        __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int ldh,
                        __nv_bfloat16* __restrict__ thi, __nv_bfloat16* __restrict__ tlo, int ldt,
                        int Mt) {
  __shared__ __nv_bfloat16 sh[32][33], sl[32][33];
  const int k0 = blockIdx.x * 32, mb = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int m = mb + i, k = k0 + threadIdx.x;
    const float v = (m < M && k < K) ? X[(int64_t)m * ldx + k] : 0.0f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    if (m < M && k < ldh) {
      hi[(int64_t)m * ldh + k] = h;
      lo[(int64_t)m * ldh + k] = l;
    }
    sh[i][threadIdx.x] = h;
    sl[i][threadIdx.x] = l;
  }
  if (!thi) return;
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int k = k0 + i, m = mb + threadIdx.x;
    if (k < K && m < Mt) {
      thi[(int64_t)k * ldt + m] = sh[threadIdx.x][i];
      tlo[(int64_t)k * ldt + m] = sl[threadIdx.x][i];
    }
  }
}

// W [K][N] (FP32) -> Wt [N][ldt] = bf16(W)^T (zero for k >= K, k < ldt) and
// Wk [K][ldk] = bf16(W) (zero for n >= N, n < ldk)
__global__ void k_weights(const float* __restrict__ W, int K, int N,
                          __nv_bfloat16* __restrict__ Wt, int ldt, __nv_bfloat16* __restrict__ Wk,
                          int ldk) {
  __shared__ __nv_bfloat16 t[32][33];
  const int n0 = blockIdx.x * 32, kb = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int k = kb + i, n = n0 + threadIdx.x;
    const __nv_bfloat16 v = __float2bfloat16_rn((k < K && n < N) ? W[(int64_t)k * N + n] : 0.0f);
    if (k < K && n < ldk) Wk[(int64_t)k * ldk + n] = v;
    t[i][threadIdx.x] = v;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int n = n0 + i, k = kb + threadIdx.x;
    if (n < N && k < ldt) Wt[(int64_t)n * ldt + k] = t[threadIdx.x][i];
  }
}

}  // namespace

cudaError_t split(const float* X, int M, int K, int ldx, __nv_bfloat16* hi, __nv_bfloat16* lo,
                  int ldh, __nv_bfloat16* thi, __nv_bfloat16* tlo, int ldt, int Mt,
                  cudaStream_t s) {
  const int kc = ldh > K ? ldh : K;
  const int mr = Mt > M ? Mt : M;
  dim3 grid((kc + 31) / 32, (mr + 31) / 32);
  k_split<<<grid, dim3(32, 8), 0, s>>>(X, M, K, ldx, hi, lo, ldh, thi, tlo, ldt, Mt);
  count_launch();
  return cudaGetLastError();
}

cudaError_t weights_bf16(const float* W, int K, int N, __nv_bfloat16* Wt, int ldt,
                         __nv_bfloat16* Wk, int ldk, cudaStream_t s) {
  const int nc = ldk > N ? ldk : N;
  const int kr = ldt > K ? ldt : K;
  dim3 grid((nc + 31) / 32, (kr + 31) / 32);
  k_weights<<<grid, dim3(32, 8), 0, s>>>(W, K, N, Wt, ldt, Wk, ldk);
  count_launch();
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace tpp
