// Internal definitions shared by the libtpp translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "tpp.h"

#define TPP_MAX_N 32
#define TPP_MAX_N_3D 16
#define TPP_MAX_MU 64

namespace tpp {

// 1D tables of the nodal basis (Sec. 3.2): Gauss-Legendre nodes x and weights
// w on [0, 1], D[a*n + j] = phi_j'(x_a), l0[j] = phi_j(0), l1[j] = phi_j(1).
struct Tables {
  double x[TPP_MAX_N];
  double w[TPP_MAX_N];
  double l0[TPP_MAX_N];
  double l1[TPP_MAX_N];
  double D[TPP_MAX_N * TPP_MAX_N];
  // float copies (rounded to nearest) for the FP32 kernels, which then issue no
  // FP64 conversion instructions
  float wf[TPP_MAX_N];
  float l0f[TPP_MAX_N];
  float l1f[TPP_MAX_N];
  float Df[TPP_MAX_N * TPP_MAX_N];
};

template <typename VT> struct Tab;
template <> struct Tab<double> {
  static __device__ const double* w(const Tables* T) { return T->w; }
  static __device__ const double* l0(const Tables* T) { return T->l0; }
  static __device__ const double* l1(const Tables* T) { return T->l1; }
  static __device__ const double* D(const Tables* T) { return T->D; }
};
template <> struct Tab<float> {
  static __device__ const float* w(const Tables* T) { return T->wf; }
  static __device__ const float* l0(const Tables* T) { return T->l0f; }
  static __device__ const float* l1(const Tables* T) { return T->l1f; }
  static __device__ const float* D(const Tables* T) { return T->Df; }
};

// Device-side status words written by kernels (never trap).
struct DevStatus {
  int32_t build_singular;   // elements whose inverted factors were singular
  int32_t build_schur_fail; // elements whose Francis iteration hit the cap
  int32_t build_schur_relaxed;  // elements deflated at sqrt(eps) (nearly defective clusters)
  int32_t build_shifted;
  int32_t build_rank1;
  double max_cond;          // stored as ordered bits via atomicMax on long long
  double min_sigma_ratio;
  int32_t nan_seen;
  int32_t z_unconverged;    // 3D stage 1: elements whose Lanczos hit its step cap
  int32_t learned_fallback; // learned build: elements handed to the exact KSVD
  int32_t mass_unconverged; // element mass solves that hit their iteration limit
  double max_cond_z;        // 3D stage 1: largest cond_1(A1)
};

// GMRES device state (one solve at a time per context).
struct GmresState {
  int32_t j;          // current Arnoldi column
  int32_t done;       // 1 when the current cycle must stop
  int32_t k;          // columns completed in this cycle
  int32_t breakdown;
  double bnorm;
  double beta;        // ||r0|| of the cycle
  double est;         // |g_{k}| / ||b||
  double rtol;
  int32_t m;          // restart length
  int32_t inner_total;   // inner FP32 steps taken in this solve (mixed mode)
  unsigned int tickets[4];   // last-block-done counters of the reduction kernels
  int32_t skip_re;    // 1: the current column needs no second Gram-Schmidt pass (or is done)
  int32_t pad3;
};

struct Layout {
  // offsets in bytes from workspace start
  size_t tables, status, gstate;
  size_t zd, rz, qo, qr_work, qr_tau;   // structure basis of the rearranged block (2D)
  size_t cx, cy, cz;                    // flux Jacobians at the volume nodes (scaled)
  size_t mq;                            // curved elements: w |J_T| at the quadrature points
  size_t fa;                            // a.n_outward at the face nodes (scaled), [E][2d][nfl]
  size_t nbr;                           // neighbour across each face, [E][2d] (-1: none)
  size_t traces;
  size_t sigma, fA1, fB1, fA2, fB2;
  size_t fSA, fSB, fQ1, fQ2, fT1, fT2, fSC;  // fSC: 3D A1^-1 factor
  size_t flags, masks;
  size_t bscr, biscr;                  // factor-build scratch (Lanczos bases, tridiagonal work)
  size_t kco;                          // per-block KSVD coefficients (Cx, Cy, Dg)
  size_t fG;                           // one-sided form: shifted inverses, 2 n^3 per element
  size_t lx, lout, lmn, lnorm, lloss, lmask;   // learned build: inputs, outputs, cores, flags
  size_t opf;                          // mixed mode: FP32 operator data (OpF32Layout)
  size_t gstate_in, gbuf_in, vi, tf;   // mixed mode: inner FP32 GMRES state, H, basis, temp
  size_t s1scr, fAz, fAzi, sigz, zflags;   // 3D stage 1: scratch, A1, A1^-1, sigma_1, flags
  size_t f32;                          // float copies of SA,SB,Q1,Q2,T1,T2 (mixed)
  size_t bj_lu, bj_piv;
  size_t tvec;                         // time integration: 6 solution-sized vectors
  size_t mtab;                         // mass solve: mu-point rule and interpolation matrix
  size_t bf16;                         // BF16 copies of the one-sided apply factors
  size_t mutab, qb, rb, qtr, bwork;    // over-integration: rule, core basis Q, R, traces, QR work
  size_t V, Z, vtmp, vtmp2, partials, hbuf, gbuf;
  size_t total;
};

// full multi-component blocks of a 2D system context (k_full.cu): workspace offsets
struct FullOffsets {
  size_t QB = 0, RB = 0, rk = 0, GB = 0, A = 0, B = 0, sig = 0, T = 0, Q = 0, Mb = 0, inv = 0,
         flags = 0, lu = 0, piv = 0, total = 0;
};

}  // namespace tpp

struct tpp_ctx {
  tpp_problem prob;        // copy (array pointers cleared: the workspace holds the data)
  int32_t n, dim;
  int32_t device;          // CUDA device the context (and its workspace) was created on
  int64_t E, N;            // elements, DOFs
  int32_t R;               // right-hand sides per element ([E][R][n^d] vectors)
  int64_t EB;              // vector blocks: E * R
  int32_t nloc;            // n^dim
  int32_t mu;              // quadrature points per direction (n: collocated; > n: over-integrated)
  int32_t nq;              // mu^dim quadrature points per element
  int32_t nfq;             // mu^(dim-1) quadrature points per face
  int32_t max_restart;
  uint32_t features;
  int32_t rz;              // rank of the off-diagonal structure block
  int32_t r;               // size of the core matrix M = n + rz
  char* ws;
  size_t ws_bytes;
  tpp::Layout L;
  bool factors_built;
  bool bj_built;
  bool isolated;           // no neighbour coupling (every nbr entry -1): block-diagonal
  bool curved = false;     // tpp_set_metric_terms: per-point mass L.mq (general geometry)
  // coupled system (k_system.cu): sys_nc components per physical element, the context's
  // elements are the (element, component) pairs; 0 for a scalar problem
  int32_t sys_nc = 0;
  int64_t sys_E = 0;
  size_t sys_cx = 0, sys_cy = 0, sys_cz = 0, sys_fo = 0, sys_fn = 0, sys_nbr = 0;
  // TPP_FEAT_FULL_BLOCKS: factors of the whole n_c n^2 blocks (and their exact LU with
  // TPP_FEAT_BLOCK_JACOBI) replace the small-block ones
  bool sys_full = false, sys_full_bj = false;
  tpp::FullOffsets fb;
  int32_t partial_blocks;  // number of CTAs of the reduction kernels
  cudaGraphExec_t gexec[64];   // use_graph: captured Arnoldi step groups, by first step
  int32_t gkernels[64];        // kernels in each (added to the launch count per replay)
  double gkey[6];              // GMRES options they were captured for
  cudaStream_t gstream;        // stream they are captured on (created at the first capture)
  template <typename T> T* p(size_t off) const { return reinterpret_cast<T*>(ws + off); }
};

namespace tpp {

void set_error(const std::string& msg);
// Number of kernels this library has launched (all threads, since load).
void count_launch(int k = 1);
tpp_status cuda_check(cudaError_t e, const char* what);

// kernels launchers (defined in the .cu files)
cudaError_t launch_tables(const tpp_ctx* c, cudaStream_t s);
cudaError_t launch_struct_qr(const tpp_ctx* c, cudaStream_t s);
// flux Jacobians from the caller's velocity arrays (NULL: a zero field)
cudaError_t launch_precompute(const tpp_ctx* c, const double* vel_nodes,
                              const double* vel_face_normal, cudaStream_t s);
cudaError_t launch_traces(const tpp_ctx* c, const double* x, double* tr, cudaStream_t s,
                          const int32_t* skip = nullptr);
cudaError_t launch_dg_apply(const tpp_ctx* c, const double* x, const double* tr, double* y,
                            const int32_t* skip, cudaStream_t s);
// curved elements: mass and flux coefficients from the caller's metric terms (2D)
cudaError_t launch_metric_2d(const tpp_ctx* c, const double* jdet, const double* flux,
                             const double* ff, double dt, cudaStream_t s);
// coupled-system operator (k_system.cu); traces tr of x per (element, component) block
cudaError_t launch_sys_apply(const tpp_ctx* c, const double* x, const double* tr, double* y,
                             const int32_t* skip, cudaStream_t s, double mass);
// full multi-component blocks (k_full.cu); the layout returns its end offset
size_t full_layout(size_t base, int dim, int n, int64_t E, bool bj, FullOffsets* out);
cudaError_t launch_full_basis(const tpp_ctx* c, cudaStream_t s);
// build steps after the KSVD: factor inverses, Schur forms, shifted inverses, S_A / S_B
// (k_build.cu), on the c->E factor sets in the workspace
cudaError_t launch_factor_inverse(const tpp_ctx* c, cudaStream_t s);
cudaError_t launch_full_build(const tpp_ctx* c, cudaStream_t s);
cudaError_t launch_full3_build(const tpp_ctx* c, cudaStream_t s);
cudaError_t launch_full3_apply(const tpp_ctx* c, const double* b, double* x, const int32_t* skip,
                               cudaStream_t s);
cudaError_t launch_full_apply(const tpp_ctx* c, const double* b, double* x, const int32_t* skip,
                              cudaStream_t s);
cudaError_t launch_full_bj_build(const tpp_ctx* c, cudaStream_t s);
cudaError_t launch_full_bj_apply(const tpp_ctx* c, const double* b, double* x,
                                 const int32_t* skip, cudaStream_t s);
// dense LU with partial pivoting of nblk row-major nb x nb blocks, and the solves
cudaError_t launch_bj_lu(int nb, int64_t nblk, double* LU, int32_t* piv, cudaStream_t s);
cudaError_t launch_bj_solve(int nb, int64_t nblk, int R, const double* LU, const int32_t* piv,
                            const double* b, double* x, const int32_t* skip, cudaStream_t s);
// over-integration (mu > n, 2D; k_overint.cu)
struct MuTables {        // the mu-point rule and the nodal basis at its points
  double x[TPP_MAX_MU], w[TPP_MAX_MU];
  double G[TPP_MAX_MU * TPP_MAX_N];      // G[a * n + j] = phi_j(x_a)
  double D[TPP_MAX_MU * TPP_MAX_N];      // D[a * n + j] = phi_j'(x_a)
  float Gf[TPP_MAX_MU * TPP_MAX_N], Df[TPP_MAX_MU * TPP_MAX_N], wf[TPP_MAX_N];
};
inline int core_size_mu(int n, int mu) {
  const int m = 2 * mu + 2;
  return (n * n < m) ? n * n : m;
}
cudaError_t launch_mu_setup(const tpp_ctx* c, cudaStream_t s);   // rule, basis QR
cudaError_t launch_core_mu(const tpp_ctx* c, cudaStream_t s);    // explicit cores R K R^T
cudaError_t launch_traces_mu(const tpp_ctx* c, const double* x, double* tr, cudaStream_t s,
                             const int32_t* skip);
cudaError_t launch_dg_apply_mu(const tpp_ctx* c, const double* x, const double* tr, double* y,
                               const int32_t* skip, cudaStream_t s, double mass);
cudaError_t launch_traces_mu_f32(const tpp_ctx* c, const float* x, float* tr, cudaStream_t s,
                                 const int32_t* skip);
cudaError_t launch_dg_apply_mu_f32(const tpp_ctx* c, const float* x, const float* tr, float* y,
                                   const int32_t* skip, cudaStream_t s);
// y = dt A x without the mass term (explicit time stepping: J x = -y / dt)
cudaError_t launch_dg_apply_flux(const tpp_ctx* c, const double* x, const double* tr, double* y,
                                 cudaStream_t s);
cudaError_t launch_build_2d(const tpp_ctx* c, cudaStream_t s);
// per-element scratch of the 3D stage-1 kernel (doubles)
struct S1Layout {
  size_t cx3, cy3, cz3, rx, ry, sd, P, Q, ut, zu, yu, wv, cw, tmp, al, be, y, d, du, du2, dl, pv,
      total;
};

__host__ __device__ inline S1Layout s1_layout(int n, int rz, int Jmax) {
  const size_t nn = (size_t)n * n, n3 = nn * n, nc = n + 2;
  S1Layout L;
  size_t o = 0;
  L.cx3 = o; o += nc * nn;
  L.cy3 = o; o += nc * nn;
  L.cz3 = o; o += nc * nn;
  L.rx = o; o += (size_t)rz * nn;
  L.ry = o; o += (size_t)rz * nn;
  L.sd = o; o += n3;
  L.P = o; o += nn;
  L.Q = o; o += (size_t)(Jmax + 1) * nn;
  L.ut = o; o += n;
  L.zu = o; o += nc;
  L.yu = o; o += nn;
  L.wv = o; o += nn;
  L.cw = o; o += nc;
  L.tmp = o; o += nn;
  L.al = o; o += Jmax + 1;
  L.be = o; o += Jmax + 2;
  L.y = o; o += Jmax + 1;
  L.d = o; o += Jmax + 1;
  L.du = o; o += Jmax + 1;
  L.du2 = o; o += Jmax + 1;
  L.dl = o; o += Jmax + 1;
  L.pv = o; o += Jmax + 1;
  L.total = (o + 3) & ~size_t(3);
  return L;
}

// Lanczos steps allowed in the 3D stage 1 (the Gram operator has order n^2)
__host__ __device__ inline int s1_jmax(int n) { return (n * n < 64) ? n * n : 64; }

cudaError_t launch_build_3d(const tpp_ctx* c, cudaStream_t s);
cudaError_t launch_ksvd_pipeline(const tpp_ctx* c, cudaStream_t s, const int32_t* mask);
cudaError_t launch_learned_inputs(const tpp_ctx* c, float* X, double* Mn, double* norms,
                                  cudaStream_t s);
cudaError_t launch_learned_accept(const tpp_ctx* c, const float* out, const double* norms,
                                  const double* lossv, double threshold, int32_t* mask,
                                  cudaStream_t s);
void mlp_forward(tpp_mlp* net, const float* X, int B, float* out, cudaStream_t s);
// error word of the network's tensor-core GEMMs (synchronises s): 0 = no pipeline wait gave up
int mlp_read_error(const tpp_mlp* net, cudaStream_t s);
size_t ksvd_scr_doubles(int n, int rz);   // KSVD scratch per element (doubles)
int mlp_n(const tpp_mlp* net);
int mlp_max_batch(const tpp_mlp* net);
cudaError_t mlp_factor_loss(const float* out, const double* Mn, const double* Qo, int n, int rz,
                            int B, float inv_batch, float* dout, double* lossv, cudaStream_t s);
cudaError_t launch_traces_f32(const tpp_ctx* c, const float* x, float* tr, cudaStream_t s,
                              const int32_t* skip);
cudaError_t launch_dg_apply_f32(const tpp_ctx* c, const float* x, const float* tr, float* y,
                                const int32_t* skip, cudaStream_t s);
cudaError_t launch_op_to_f32(const tpp_ctx* c, cudaStream_t s);
cudaError_t launch_apply_f32(const tpp_ctx* c, const float* b, float* x, const int32_t* skip,
                             cudaStream_t s);
// float32 copies of the apply factors (offsets in floats from Layout::f32)
struct F32Layout {
  size_t SA, SB, Q1, Q2, T1, T2, Azi, G, total;
};
inline F32Layout f32_layout(int n, int64_t E, int dim, bool two) {
  const size_t m = (size_t)E * n * n;
  F32Layout L{};
  size_t o = 0;
  L.SA = o; o += m;
  L.SB = o; o += m;
  L.Q1 = o; o += m;
  L.T1 = o; o += m;
  if (two) { L.Q2 = o; o += m; L.T2 = o; o += m; }
  if (dim == 3) { L.Azi = o; o += m; }
  if (!two) { L.G = o; o += 2 * m * n; }
  L.total = o;
  return L;
}

// float copies of the operator data for the FP32 inner solves (offsets in
// floats from Layout::opf): volume coefficients (E n^d each), face coefficients
// (E 2d n^(d-1)), face traces (EB 2d n^(d-1))
struct OpF32Layout {
  size_t cx, cy, cz, fa, tr, mq, total;
};
inline OpF32Layout op_f32_layout(int dim, int64_t Nc, int64_t E, int n, int64_t EB) {
  const size_t nfl = (dim == 2) ? (size_t)n : (size_t)n * n;   // n: points per direction
  OpF32Layout L{};
  size_t o = 0;
  L.cx = o; o += Nc;
  L.cy = o; o += Nc;
  L.cz = o; if (dim == 3) o += Nc;
  L.fa = o; o += E * 2 * dim * nfl;
  L.tr = o; o += EB * 2 * dim * nfl;
  L.mq = o; o += Nc;
  L.total = o;
  return L;
}
inline OpF32Layout op_f32_layout(const tpp_ctx* c) {
  return op_f32_layout(c->dim, c->E * c->nq, c->E, c->mu, c->EB);
}

// A view of the context for a call on nrhs <= R right-hand sides per element
// (vectors [E][nrhs][n^d]): the same workspace with R, EB and N of the call.
inline tpp_ctx call_view(const tpp_ctx* c, int nrhs) {
  tpp_ctx v = *c;
  v.R = nrhs;
  v.EB = c->E * nrhs;
  v.N = v.EB * c->nloc;
  return v;
}

// the paper's two-sided Schur form (both factor products reduced) instead of
// the default one-sided form with shifted inverses
inline bool two_sided(const tpp_ctx* c) { return (c->features & TPP_FEAT_TWO_SIDED) != 0; }
cudaError_t launch_apply_2d(const tpp_ctx* c, const double* b, double* x, int prec,
                            const int32_t* skip, cudaStream_t s);
cudaError_t launch_apply_3d(const tpp_ctx* c, const double* b, double* x, int prec,
                            const int32_t* skip, cudaStream_t s);
cudaError_t launch_to_f32(const tpp_ctx* c, cudaStream_t s);
// BF16 tensor-core apply (2D, n <= 16, one-sided form; k_apply_tc.cu)
size_t bf16_factor_bytes(int n, int64_t E);
cudaError_t launch_to_bf16(const tpp_ctx* c, cudaStream_t s);
cudaError_t launch_apply_bf16(const tpp_ctx* c, const double* b, double* x, const int32_t* skip,
                              cudaStream_t s);
cudaError_t launch_apply_bf16_f32(const tpp_ctx* c, const float* b, float* x,
                                  const int32_t* skip, cudaStream_t s);
cudaError_t launch_bj_build(const tpp_ctx* c, cudaStream_t s);
cudaError_t launch_bj_apply(const tpp_ctx* c, const double* b, double* x, const int32_t* skip,
                            cudaStream_t s);

}  // namespace tpp

// ---------------------------------------------------------------------------
// small device helpers
namespace tpp {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; `red` must hold blockDim.x/32 doubles.  All threads get the result.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += red[i];   // same order in every thread: deterministic
  return t;
}

// k-th (ascending) Gauss-Legendre node and weight of the n-point rule on [0, 1]:
// Newton's method on the three-term Legendre recurrence from cos(pi (j + 3/4) /
// (n + 1/2)), j = n - 1 - k; weight 1 / ((1 - t^2) P_n'(t)^2) on [0, 1].
__device__ inline void gauss_legendre_node(int n, int k, double* node, double* weight) {
  const int jj = n - 1 - k;
  double x = cos(M_PI * (jj + 0.75) / (n + 0.5));
  double dp = 1.0;
  for (int it = 0; it < 100; ++it) {
    double p0 = 1.0, p1 = x;
    for (int m = 2; m <= n; ++m) {
      const double p2 = ((2.0 * m - 1.0) * x * p1 - (m - 1.0) * p0) / m;
      p0 = p1;
      p1 = p2;
    }
    const double pn = (n == 1) ? x : p1;
    const double pm = (n == 1) ? 1.0 : p0;
    dp = n * (x * pn - pm) / (x * x - 1.0);
    const double dx = pn / dp;
    x -= dx;
    if (fabs(dx) <= 1e-16 * fmax(1.0, fabs(x))) break;
  }
  double p0 = 1.0, p1 = x;
  for (int m = 2; m <= n; ++m) {
    const double p2 = ((2.0 * m - 1.0) * x * p1 - (m - 1.0) * p0) / m;
    p0 = p1;
    p1 = p2;
  }
  const double pn = (n == 1) ? x : p1;
  const double pm = (n == 1) ? 1.0 : p0;
  dp = n * (x * pn - pm) / (x * x - 1.0);
  *node = 0.5 * (x + 1.0);
  *weight = 1.0 / ((1.0 - x * x) * dp * dp);
}

// SplitMix64 (Steele, Lea & Flood 2014) mapped to [-1, 1): deterministic
// "random" start vectors for the Lanczos iteration.
__device__ __forceinline__ double splitmix_unit(uint64_t salt, uint64_t i) {
  uint64_t z = salt * 0x9E3779B97F4A7C15ull + (i + 1) * 0xBF58476D1CE4E5B9ull;
  z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27; z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

}  // namespace tpp
