// Host side of the C ABI declared in include/tpp.h: validation, workspace
// layout, launch sequencing and the restarted GMRES driver.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>
#include <atomic>

#include "tpp_internal.cuh"

namespace tpp {

static thread_local std::string g_last_error = "no error";

void set_error(const std::string& msg) { g_last_error = msg; }

static std::atomic<long long> g_launches{0};
void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

tpp_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TPP_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return TPP_ERR_CUDA;
}

// GMRES kernels (k_gmres.cu)
template <typename VT>
cudaError_t gmres_dots(const VT* V, int64_t N, int nvec, const VT* w, double* partials,
                       int stride, int nblk, const int32_t* skip, double* h_out,
                       unsigned int* ticket, cudaStream_t s);
template <typename VT>
cudaError_t gmres_update(const VT* V, int64_t N, int nvec, const double* h, VT* w,
                         double* partials, int stride, int mode, int nblk, const int32_t* skip,
                         double* h_out, unsigned int* ticket, GmresState* st, double* H,
                         double* cs, double* sn, double* g, double* h1, double* h2,
                         double* inv_beta, int j, cudaStream_t s);
cudaError_t gmres_lsq(const GmresState* st, const double* H, const double* g, double* y,
                      cudaStream_t s);
cudaError_t gmres_combine(const double* B, int64_t N, const GmresState* st, const double* y,
                          double* out, int accumulate, cudaStream_t s);
cudaError_t gmres_combine_f32(const float* B, int64_t N, const GmresState* st, const double* y,
                              double* out, const int32_t* skip, cudaStream_t s);
cudaError_t vec_scale(double* out, const double* in, int64_t N, const double* sptr, double sval,
                      const int32_t* skip, cudaStream_t s);
cudaError_t vec_scale_f32(float* out, const float* in, int64_t N, const double* sptr,
                          double sval, const int32_t* skip, cudaStream_t s);
cudaError_t vec_to_float(const double* in, float* out, int64_t N, const int32_t* skip,
                         cudaStream_t s);
cudaError_t vec_sub(double* out, const double* a, const double* b, int64_t N, cudaStream_t s);
cudaError_t vec_norm(const double* x, int64_t N, double* partials, int stride, int nblk,
                     double* out, cudaStream_t s);
cudaError_t gmres_cycle_init(GmresState* st, double* g, double beta, int m, double bnorm,
                             double rtol, const int32_t* done_src, cudaStream_t s);
cudaError_t vec_axpy(double* out, const double* in, double a, int64_t N, cudaStream_t s);
cudaError_t accumulate_inner(GmresState* outer, const GmresState* inner, const int32_t* skip,
                             cudaStream_t s);

namespace {

constexpr int kPartialBlocks = 152 * 4;
constexpr int kPartialStride = 64;
constexpr int kMaxRestart = 63;
constexpr int kLookahead = 8;     // Arnoldi steps enqueued between host reads of the state

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct GBuf {   // offsets (doubles) inside the gbuf region
  size_t H, cs, sn, g, h1, h2, y, invb, scal, total;
};

GBuf gbuf_layout(int m) {
  GBuf b;
  b.H = 0;
  b.cs = b.H + (size_t)(m + 1) * m;
  b.sn = b.cs + m;
  b.g = b.sn + m;
  b.h1 = b.g + m + 1;
  b.h2 = b.h1 + m + 1;
  b.y = b.h2 + m + 1;
  b.invb = b.y + m;
  b.scal = b.invb + 1;
  b.total = b.scal + 8;
  return b;
}

const char* validate(const tpp_problem* p, int32_t max_restart) {
  if (!p) return "problem is NULL";
  if (p->dim != 2 && p->dim != 3) return "dim must be 2 or 3";
  if (p->n < 1 || p->n > TPP_MAX_N) return "n must be in [1, 32]";
  if (p->dim == 3 && p->n > TPP_MAX_N_3D) return "n must be in [1, 16] in 3D";
  if (p->num_elem < 1 || p->num_elem > (int64_t)INT32_MAX) return "num_elem must be in [1, 2^31)";
  if (p->nrhs < 1) return "nrhs must be >= 1";
  if ((int64_t)p->num_elem * p->nrhs > (int64_t)INT32_MAX)
    return "num_elem * nrhs must be below 2^31";
  if (!(p->h > 0.0) || !std::isfinite(p->h)) return "h must be positive and finite";
  if (!(p->dt >= 0.0) || !std::isfinite(p->dt)) return "dt must be >= 0 and finite";
  if (max_restart < 1 || max_restart > kMaxRestart) return "max_restart must be in [1, 63]";
  if (p->mu != 0 && (p->mu < p->n || p->mu > TPP_MAX_MU)) return "mu must be 0 or in [n, 64]";
  if (p->mu > p->n && p->dim != 2) return "over-integration (mu > n) is implemented in 2D";
  if (p->mu > p->n && p->mu > 32)
    return "over-integration needs mu <= 32 (KSVD core of size up to 2 mu + 2 <= 66)";
  if ((p->vel_nodes == nullptr) != (p->vel_face_normal == nullptr))
    return "vel_nodes and vel_face_normal must both be given or both be NULL";
  return nullptr;
}

Layout compute_layout(const tpp_problem* p, int32_t max_restart, uint32_t features,
                      int* rz_out) {
  const int n = p->n, d = p->dim;
  const int64_t E = p->num_elem;
  const int32_t R = p->nrhs;
  const int64_t EB = E * R;
  const int64_t nloc = (d == 2) ? (int64_t)n * n : (int64_t)n * n * n;
  const int mu = (p->mu > n) ? p->mu : n;            // quadrature points per direction
  const int64_t nfl = (d == 2) ? mu : (int64_t)mu * mu;
  const int64_t N = EB * nloc;
  const int64_t Nc = E * ((d == 2) ? (int64_t)mu * mu : (int64_t)mu * mu * mu);
  const int nc = n + 2, Ro = n * n - n;
  const int rz = Ro < nc ? Ro : nc;
  if (rz_out) *rz_out = rz;
  const int m = max_restart;
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + (bytes ? bytes : 8));
    return o;
  };
  L.tables = take(sizeof(Tables));
  L.status = take(sizeof(DevStatus));
  L.gstate = take(sizeof(GmresState));
  L.gbuf = take(gbuf_layout(m).total * sizeof(double));
  L.zd = take((size_t)n * nc * 8);
  L.rz = take((size_t)nc * nc * 8);
  L.qo = take((size_t)Ro * nc * 8);
  L.qr_work = take((size_t)Ro * nc * 8);
  L.qr_tau = take((size_t)nc * 8);
  L.cx = take((size_t)Nc * 8);
  L.cy = take((size_t)Nc * 8);
  L.cz = (d == 3) ? take((size_t)Nc * 8) : 0;
  L.fa = take((size_t)E * 2 * d * nfl * 8);
  L.mq = take((size_t)Nc * 8);
  L.nbr = take((size_t)E * 2 * d * 4);
  L.traces = take((size_t)EB * 2 * d * nfl * 8);
  const size_t fsz = (size_t)E * n * n * 8;
  L.sigma = take((size_t)E * 2 * 8);
  L.fA1 = take(fsz);
  L.fB1 = take(fsz);
  L.fA2 = take(fsz);
  L.fB2 = take(fsz);
  L.fSA = take(fsz);
  L.fSB = take(fsz);
  L.fQ1 = take(fsz);
  const bool two = (features & TPP_FEAT_TWO_SIDED) != 0;
  L.fQ2 = two ? take(fsz) : 0;
  L.fT1 = take(fsz);
  L.fT2 = take(fsz);
  L.fSC = take((size_t)E * 8);
  L.flags = take((size_t)E * 4);
  L.masks = take((size_t)E * 2 * 4);
  {
    // KSVD core size: n + rz collocated; min(n^2, 2 mu + 2) over-integrated
    const int rc = (mu > n) ? core_size_mu(n, mu) : n + rz;
    const size_t r = (size_t)rc;
    L.bscr = take((size_t)E * ksvd_scr_doubles(n, rc - n) * 8);
    L.biscr = take((size_t)E * 4 * r * 4);
    // coefficients of the 2D-structured block fed to the KSVD (2D: the element
    // block; 3D: the second-stage block D1): Cx, Cy ((n+2) x n each), Dg (n x n);
    // over-integrated: the explicit cores (r x r)
    const size_t per = (mu > n) ? r * r : (2 * (size_t)nc * n + (size_t)n * n);
    L.kco = take((size_t)E * per * 8);
  }
  if (mu > n) {
    const int m = 2 * mu + 2, rc = core_size_mu(n, mu);
    L.mutab = take(sizeof(MuTables));
    L.qb = take((size_t)n * n * rc * 8);
    L.rb = take((size_t)rc * m * 8);
    L.qtr = take((size_t)rc * 8);
    L.bwork = take((size_t)n * n * m * 8 + (size_t)m * 8);
  }
  if (d == 3) {
    L.s1scr = take((size_t)E * s1_layout(n, rz, s1_jmax(n)).total * 8);
    L.fAz = take(fsz);
    L.fAzi = take(fsz);
    L.sigz = take((size_t)E * 8);
    L.zflags = take((size_t)E * 4);
  }
  // the one-sided shifted inverses (2 n^3 doubles per element); with TPP_FEAT_F32_SHIFTS
  // they exist only as the FP32 copies
  L.fG = (two || (features & TPP_FEAT_F32_SHIFTS)) ? 0 : take(fsz * 2 * n);
  if (features & TPP_FEAT_LEARNED) {
    const size_t r = (size_t)n + rz;
    L.lx = take((size_t)E * (2 * n * n + 1) * 4);
    L.lout = take((size_t)E * 4 * n * n * 4);
    L.lmn = take((size_t)E * r * r * 8);
    L.lnorm = take((size_t)E * 8);
    L.lloss = take((size_t)E * 8);
    L.lmask = take((size_t)E * 4);
  }
  L.f32 = (features & TPP_FEAT_MIXED) ? take(f32_layout(n, E, d, two).total * 4) : 0;
  if (features & TPP_FEAT_MIXED) {      // FP32 operator and inner GMRES
    L.opf = take(op_f32_layout(d, Nc, E, mu, EB).total * 4);
    L.gstate_in = take(sizeof(GmresState));
    L.gbuf_in = take(gbuf_layout(m).total * sizeof(double));
    L.vi = take((size_t)(m + 1) * N * 4);
    L.tf = take((size_t)N * 4);
  }
  L.bj_lu = (features & TPP_FEAT_BLOCK_JACOBI) ? take((size_t)E * nloc * nloc * 8) : 0;
  L.bj_piv = (features & TPP_FEAT_BLOCK_JACOBI) ? take((size_t)E * nloc * 4) : 0;
  L.tvec = (features & TPP_FEAT_TIME) ? take((size_t)6 * N * 8) : 0;
  L.mtab = take((size_t)(2 * TPP_MAX_MU + TPP_MAX_MU * TPP_MAX_N) * 8);
  L.bf16 = (features & TPP_FEAT_BF16) ? take(bf16_factor_bytes(n, E)) : 0;
  L.V = take((size_t)(m + 1) * N * 8);
  L.Z = take((size_t)m * N * 8);
  L.vtmp = take((size_t)N * 8);
  L.vtmp2 = take((size_t)N * 8);
  L.partials = take((size_t)kPartialBlocks * kPartialStride * 8);
  L.hbuf = 0;
  L.total = off;
  return L;
}

#define TPP_TRY_CUDA(expr, what)                          \
  do {                                                    \
    tpp_status _s = cuda_check((expr), what);             \
    if (_s != TPP_OK) return _s;                          \
  } while (0)

tpp_status check_ctx(const tpp_ctx* c) {
  if (!c) {
    set_error("context is NULL");
    return TPP_ERR_INVALID_ARG;
  }
  return TPP_OK;
}

DevStatus fresh_status() {
  DevStatus st;
  std::memset(&st, 0, sizeof(st));
  st.max_cond = 0.0;
  st.min_sigma_ratio = 1.0;
  return st;
}

// y = S x through the sum-factorised operator (traces then element kernel)
cudaError_t apply_operator(const tpp_ctx* c, const double* x, double* y, const int32_t* skip,
                           cudaStream_t s) {
  cudaError_t e = launch_traces(c, x, c->p<double>(c->L.traces), s);
  if (e != cudaSuccess) return e;
  return launch_dg_apply(c, x, c->p<double>(c->L.traces), y, skip, s);
}

cudaError_t apply_precond(const tpp_ctx* c, int pc, int prec, const double* b, double* x,
                          const int32_t* skip, cudaStream_t s) {
  if (pc == TPP_PC_NONE) {
    return cudaMemcpyAsync(x, b, (size_t)c->N * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  if (c->sys_full) {
    if (pc == TPP_PC_BLOCK_JACOBI) return launch_full_bj_apply(c, b, x, skip, s);
    return c->dim == 2 ? launch_full_apply(c, b, x, skip, s) : launch_full3_apply(c, b, x, skip, s);
  }
  if (pc == TPP_PC_BLOCK_JACOBI) return launch_bj_apply(c, b, x, skip, s);
  if (prec == TPP_BF16) return launch_apply_bf16(c, b, x, skip, s);
  if (c->dim == 2) return launch_apply_2d(c, b, x, prec, skip, s);
  return launch_apply_3d(c, b, x, prec, skip, s);
}

}  // namespace
}  // namespace tpp

using namespace tpp;

namespace {
// TPP_FEAT_F32_SHIFTS: the shifted inverses of the one-sided form in FP32 only, for the
// FP32 apply of the mixed-precision solver
const char* f32_shifts_invalid(const tpp_problem* prob, uint32_t features) {
  if (!(features & TPP_FEAT_F32_SHIFTS)) return nullptr;
  if (!(features & TPP_FEAT_MIXED) || (features & (TPP_FEAT_TWO_SIDED | TPP_FEAT_BF16 |
                                                   TPP_FEAT_TIME | TPP_FEAT_LEARNED)) ||
      prob->n > 16 || prob->mu > prob->n)
    return "TPP_FEAT_F32_SHIFTS needs TPP_FEAT_MIXED and the one-sided form, n <= 16, mu <= n, "
           "and excludes TPP_FEAT_BF16, TPP_FEAT_TIME and TPP_FEAT_LEARNED";
  return nullptr;
}
}  // namespace

extern "C" {

const char* tpp_last_error(void) { return g_last_error.c_str(); }

int64_t tpp_kernel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

size_t tpp_workspace_bytes(const tpp_problem* prob, int32_t max_restart, uint32_t features) {
  if (validate(prob, max_restart)) return 0;
  if (const char* why = f32_shifts_invalid(prob, features)) {
    set_error(why);
    return 0;
  }
  return compute_layout(prob, max_restart, features, nullptr).total;
}

tpp_status tpp_create(tpp_ctx** out, const tpp_problem* prob, int32_t max_restart,
                      uint32_t features, void* workspace, size_t ws_bytes, void* stream) {
  if (!out) {
    set_error("out is NULL");
    return TPP_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (const char* why = validate(prob, max_restart)) {
    set_error(why);
    return TPP_ERR_INVALID_ARG;
  }
  if (prob->dim == 3 && (features & TPP_FEAT_LEARNED)) {
    set_error("learned factors are implemented for 2D problems only");
    return TPP_ERR_UNSUPPORTED;
  }
  if ((features & TPP_FEAT_BF16) &&
      (prob->dim != 2 || prob->n > 16 || (features & TPP_FEAT_TWO_SIDED))) {
    set_error("the BF16 tensor-core apply is implemented for 2D, n <= 16, one-sided form");
    return TPP_ERR_UNSUPPORTED;
  }
  if (const char* why = f32_shifts_invalid(prob, features)) {
    set_error(why);
    return TPP_ERR_INVALID_ARG;
  }
  if (prob->mu > prob->n &&
      (features & (TPP_FEAT_BLOCK_JACOBI | TPP_FEAT_LEARNED | TPP_FEAT_TIME | TPP_FEAT_BF16))) {
    set_error("over-integration (mu > n) does not support block Jacobi, learned factors, time "
              "integration (its mass matrix is not diagonal) or the BF16 apply");
    return TPP_ERR_UNSUPPORTED;
  }
  if (!prob->nbr) {
    set_error("nbr is NULL");
    return TPP_ERR_INVALID_ARG;
  }
  int rz = 0;
  const Layout L = compute_layout(prob, max_restart, features, &rz);
  if (!workspace || ws_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255u)) {
    set_error("workspace NULL, smaller than tpp_workspace_bytes() or not 256-byte aligned");
    return TPP_ERR_WORKSPACE;
  }
  int dev = 0;
  TPP_TRY_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  cudaPointerAttributes attr;
  TPP_TRY_CUDA(cudaPointerGetAttributes(&attr, workspace), "cudaPointerGetAttributes");
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) {
    set_error("workspace is not device memory");
    return TPP_ERR_INVALID_ARG;
  }
  // connectivity: checked on the host, then kept in the workspace
  const int nface = 2 * prob->dim;
  std::vector<int32_t> nb((size_t)prob->num_elem * nface);
  TPP_TRY_CUDA(cudaMemcpy(nb.data(), prob->nbr, nb.size() * sizeof(int32_t), cudaMemcpyDefault),
               "read nbr");
  for (size_t i = 0; i < nb.size(); ++i)
    if (nb[i] < -1 || nb[i] >= prob->num_elem) {
      set_error("nbr entry " + std::to_string(i) + " = " + std::to_string(nb[i]) +
                " is outside [-1, num_elem)");
      return TPP_ERR_INVALID_ARG;
    }
  tpp_ctx* c = new tpp_ctx();
  c->isolated = std::all_of(nb.begin(), nb.end(), [](int32_t v) { return v == -1; });
  c->prob = *prob;
  c->prob.vel_nodes = nullptr;
  c->prob.vel_face_normal = nullptr;
  c->prob.nbr = nullptr;
  c->n = prob->n;
  c->dim = prob->dim;
  c->device = dev;
  c->E = prob->num_elem;
  c->R = prob->nrhs;
  c->EB = c->E * c->R;
  c->nloc = (prob->dim == 2) ? prob->n * prob->n : prob->n * prob->n * prob->n;
  c->N = c->EB * c->nloc;
  c->mu = (prob->mu > prob->n) ? prob->mu : prob->n;
  c->nq = (prob->dim == 2) ? c->mu * c->mu : c->mu * c->mu * c->mu;
  c->nfq = (prob->dim == 2) ? c->mu : c->mu * c->mu;
  c->max_restart = max_restart;
  c->features = features;
  c->rz = rz;
  c->r = (c->mu > c->n) ? core_size_mu(c->n, c->mu) : prob->n + rz;
  c->ws = static_cast<char*>(workspace);
  c->ws_bytes = ws_bytes;
  c->L = L;
  c->factors_built = false;
  c->bj_built = false;
  c->partial_blocks = kPartialBlocks;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const DevStatus st0 = fresh_status();
  tpp_status rc = TPP_OK;
  do {
    if ((rc = cuda_check(cudaMemcpyAsync(c->ws + L.nbr, nb.data(), nb.size() * sizeof(int32_t),
                                         cudaMemcpyHostToDevice, s), "copy nbr")) != TPP_OK)
      break;
    if ((rc = cuda_check(cudaMemcpyAsync(c->ws + L.status, &st0, sizeof(st0),
                                         cudaMemcpyHostToDevice, s), "init status")) != TPP_OK) break;
    if ((rc = cuda_check(cudaMemsetAsync(c->ws + L.tables, 0, sizeof(Tables), s), "memset")) != TPP_OK) break;
    if ((rc = cuda_check(cudaMemsetAsync(c->ws + L.gstate, 0, sizeof(GmresState), s), "memset")) != TPP_OK) break;
    if (L.gstate_in &&
        (rc = cuda_check(cudaMemsetAsync(c->ws + L.gstate_in, 0, sizeof(GmresState), s),
                         "memset")) != TPP_OK)
      break;
    if ((rc = cuda_check(launch_tables(c, s), "k_tables")) != TPP_OK) break;
    if ((rc = cuda_check(launch_struct_qr(c, s), "k_struct_qr")) != TPP_OK) break;
    if (c->mu > c->n && (rc = cuda_check(launch_mu_setup(c, s), "over-integration setup")) != TPP_OK)
      break;
    if ((rc = cuda_check(launch_precompute(c, prob->vel_nodes, prob->vel_face_normal, s),
                         "k_precompute")) != TPP_OK)
      break;
    if ((features & TPP_FEAT_MIXED) &&
        (rc = cuda_check(launch_op_to_f32(c, s), "k_op_to_f32")) != TPP_OK)
      break;
    if ((rc = cuda_check(cudaStreamSynchronize(s), "tpp_create sync")) != TPP_OK) break;
  } while (0);
  if (rc != TPP_OK) {
    delete c;
    return rc;
  }
  *out = c;
  return TPP_OK;
}

tpp_status tpp_set_velocity(tpp_ctx* c, const double* vel_nodes, const double* vel_face_normal,
                            double dt, void* stream) {
  if (tpp_status r = check_ctx(c)) return r;
  if (c->sys_nc > 0) {
    set_error("tpp_set_velocity: a system context's coefficients come from tpp_create_system");
    return TPP_ERR_INVALID_ARG;
  }
  if (!vel_nodes || !vel_face_normal || !(dt >= 0.0) || !std::isfinite(dt)) {
    set_error("tpp_set_velocity: vel_nodes and vel_face_normal non-NULL, dt >= 0 and finite");
    return TPP_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->prob.dt = dt;
  c->factors_built = false;
  c->bj_built = false;
  c->curved = false;
  TPP_TRY_CUDA(launch_precompute(c, vel_nodes, vel_face_normal, s), "k_precompute");
  if (c->features & TPP_FEAT_MIXED) TPP_TRY_CUDA(launch_op_to_f32(c, s), "k_op_to_f32");
  TPP_TRY_CUDA(cudaStreamSynchronize(s), "tpp_set_velocity sync");
  return TPP_OK;
}

tpp_status tpp_set_metric_terms(tpp_ctx* c, const double* jdet, const double* flux,
                                const double* flux_face, double dt, void* stream) {
  if (tpp_status r = check_ctx(c)) return r;
  if (c->dim != 2 || c->sys_nc > 0 || (c->features & TPP_FEAT_LEARNED)) {
    set_error("tpp_set_metric_terms: 2D scalar contexts without TPP_FEAT_LEARNED only");
    return TPP_ERR_UNSUPPORTED;
  }
  if (!jdet || !flux || !flux_face || !(dt >= 0.0) || !std::isfinite(dt)) {
    set_error("tpp_set_metric_terms: jdet, flux and flux_face non-NULL, dt >= 0 and finite");
    return TPP_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->prob.dt = dt;
  c->factors_built = false;
  c->bj_built = false;
  c->curved = true;
  TPP_TRY_CUDA(launch_metric_2d(c, jdet, flux, flux_face, dt, s), "k_metric_2d");
  if (c->features & TPP_FEAT_MIXED) TPP_TRY_CUDA(launch_op_to_f32(c, s), "k_op_to_f32");
  TPP_TRY_CUDA(cudaStreamSynchronize(s), "tpp_set_metric_terms sync");
  return TPP_OK;
}

tpp_status tpp_gauss_legendre(const tpp_ctx* c, double* nodes, double* weights) {
  if (tpp_status r = check_ctx(c)) return r;
  if (!nodes || !weights) {
    set_error("nodes and weights must be non-NULL");
    return TPP_ERR_INVALID_ARG;
  }
  const double* xs = c->p<Tables>(c->L.tables)->x;
  const double* ws = c->p<Tables>(c->L.tables)->w;
  if (c->mu > c->n) {
    xs = c->p<MuTables>(c->L.mutab)->x;
    ws = c->p<MuTables>(c->L.mutab)->w;
  }
  TPP_TRY_CUDA(cudaMemcpy(nodes, xs, c->mu * sizeof(double), cudaMemcpyDeviceToHost),
               "read nodes");
  TPP_TRY_CUDA(cudaMemcpy(weights, ws, c->mu * sizeof(double), cudaMemcpyDeviceToHost),
               "read weights");
  return TPP_OK;
}

void tpp_destroy(tpp_ctx* ctx) {
  if (ctx)
    for (int q = 0; q < kMaxRestart; ++q)
      if (ctx->gexec[q]) cudaGraphExecDestroy(ctx->gexec[q]);
  if (ctx && ctx->gstream) cudaStreamDestroy(ctx->gstream);
  delete ctx;
}

int64_t tpp_num_dofs(const tpp_ctx* ctx) { return ctx ? ctx->N : -1; }
int64_t tpp_num_elem(const tpp_ctx* ctx) { return ctx ? ctx->E : -1; }

namespace {
// status of the build just enqueued -> report and return code
tpp_status finish_build(tpp_ctx* c, tpp_build_report* report, cudaStream_t s) {
  if (c->features & TPP_FEAT_MIXED) TPP_TRY_CUDA(launch_to_f32(c, s), "k_to_f32");
  if (c->features & TPP_FEAT_BF16) TPP_TRY_CUDA(launch_to_bf16(c, s), "k_bf16_factors");
  DevStatus st;
  TPP_TRY_CUDA(cudaMemcpyAsync(&st, c->ws + c->L.status, sizeof(st), cudaMemcpyDeviceToHost, s),
               "read status");
  TPP_TRY_CUDA(cudaStreamSynchronize(s), "tpp_build_factors sync");
  if (report) {
    report->num_elem = (int32_t)c->E;
    report->num_shifted = st.build_shifted;
    report->num_rank1 = st.build_rank1;
    report->num_schur_fail = st.build_schur_fail;
    report->num_schur_relaxed = st.build_schur_relaxed;
    report->max_cond = st.max_cond;
    report->min_sigma_ratio = st.min_sigma_ratio;
    report->max_cond_z = st.max_cond_z;
    report->num_z_unconverged = st.z_unconverged;
    report->num_fallback = st.learned_fallback;
  }
  c->factors_built = true;
  if (st.build_schur_fail) {
    set_error("Francis QR hit its iteration cap on " + std::to_string(st.build_schur_fail) +
              " element(s)");
    return TPP_ERR_SCHUR;
  }
  if (st.build_singular) {
    set_error(std::to_string(st.build_singular) + " element(s) have singular Kronecker factors");
    return TPP_ERR_SINGULAR_FACTOR;
  }
  return TPP_OK;
}
}  // namespace

tpp_status tpp_build_factors(tpp_ctx* c, tpp_build_report* report, void* stream) {
  if (tpp_status r = check_ctx(c)) return r;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const DevStatus st0 = fresh_status();
  TPP_TRY_CUDA(cudaMemcpyAsync(c->ws + c->L.status, &st0, sizeof(st0), cudaMemcpyHostToDevice, s),
               "reset status");
  if (c->sys_full)
    TPP_TRY_CUDA(c->dim == 2 ? launch_full_build(c, s) : launch_full3_build(c, s),
                 "k_full (full-block factors)");
  else
    TPP_TRY_CUDA(c->dim == 2 ? launch_build_2d(c, s) : launch_build_3d(c, s), "k_build");
  return finish_build(c, report, s);
}

int32_t tpp_core_size(const tpp_ctx* c) { return c ? c->r : -1; }

tpp_status tpp_learned_inputs(const tpp_ctx* c, float* X, double* Mn, double* norms,
                              void* stream) {
  if (tpp_status r = check_ctx(c)) return r;
  if (c->dim != 2 || (Mn && !norms) || (!X && !Mn)) {
    set_error("tpp_learned_inputs: 2D context; Mn needs norms; X or Mn required");
    return TPP_ERR_INVALID_ARG;
  }
  TPP_TRY_CUDA(launch_learned_inputs(c, X, Mn, norms, static_cast<cudaStream_t>(stream)),
               "tpp_learned_inputs");
  return TPP_OK;
}

tpp_status tpp_build_factors_learned(tpp_ctx* c, tpp_mlp* net, double threshold,
                                     tpp_build_report* report, void* stream) {
  if (tpp_status r = check_ctx(c)) return r;
  if (!net || c->dim != 2 || !(c->features & TPP_FEAT_LEARNED) || mlp_n(net) != c->n ||
      !(threshold >= 0.0)) {
    set_error("tpp_build_factors_learned: 2D context with TPP_FEAT_LEARNED, network of the "
              "same n, threshold >= 0");
    return TPP_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const DevStatus st0 = fresh_status();
  TPP_TRY_CUDA(cudaMemcpyAsync(c->ws + c->L.status, &st0, sizeof(st0), cudaMemcpyHostToDevice, s),
               "reset status");
  float* X = c->p<float>(c->L.lx);
  float* out = c->p<float>(c->L.lout);
  double* Mn = c->p<double>(c->L.lmn);
  double* norms = c->p<double>(c->L.lnorm);
  double* lossv = c->p<double>(c->L.lloss);
  TPP_TRY_CUDA(launch_learned_inputs(c, X, Mn, norms, s), "learned inputs");
  const int n = c->n, K = 2 * n * n + 1, O = 4 * n * n, r = c->r, mb = mlp_max_batch(net);
  for (int64_t e0 = 0; e0 < c->E; e0 += mb) {
    const int B = (int)((c->E - e0) < mb ? (c->E - e0) : mb);
    mlp_forward(net, X + e0 * K, B, out + e0 * O, s);
    TPP_TRY_CUDA(mlp_factor_loss(out + e0 * O, Mn + e0 * r * r, c->p<double>(c->L.qo), n, c->rz,
                                 B, 1.0f, nullptr, lossv + e0, s), "learned loss");
  }
  TPP_TRY_CUDA(launch_learned_accept(c, out, norms, lossv, threshold, c->p<int32_t>(c->L.lmask), s),
               "learned accept");
  TPP_TRY_CUDA(launch_ksvd_pipeline(c, s, c->p<int32_t>(c->L.lmask)), "k_build (fallback)");
  const tpp_status st = finish_build(c, report, s);
  if (mlp_read_error(net, s) != 0) {
    set_error("a tensor-core GEMM of the network gave up waiting on its pipeline");
    return TPP_ERR_TIMEOUT;
  }
  return st;
}

tpp_status tpp_build_block_jacobi(tpp_ctx* c, void* stream) {
  if (tpp_status r = check_ctx(c)) return r;
  if (!(c->features & TPP_FEAT_BLOCK_JACOBI) && !c->sys_full_bj) {
    set_error("context was created without TPP_FEAT_BLOCK_JACOBI");
    return TPP_ERR_INVALID_ARG;
  }
  TPP_TRY_CUDA(c->sys_full_bj ? launch_full_bj_build(c, static_cast<cudaStream_t>(stream))
                              : launch_bj_build(c, static_cast<cudaStream_t>(stream)),
               "block Jacobi build");
  c->bj_built = true;
  return TPP_OK;
}

namespace {
tpp_status check_nrhs(const tpp_ctx* c, int32_t nrhs) {
  if (nrhs < 1 || nrhs > c->R) {
    set_error("nrhs must be in [1, the problem's nrhs = " + std::to_string(c->R) + "]");
    return TPP_ERR_INVALID_ARG;
  }
  return TPP_OK;
}
}  // namespace

tpp_status tpp_apply_inverse(const tpp_ctx* c, const double* b, double* x, int32_t nrhs,
                             int32_t prec, void* stream) {
  if (tpp_status r = check_ctx(c)) return r;
  if (tpp_status r = check_nrhs(c, nrhs)) return r;
  if (!b || !x || b == x) {
    set_error("b and x must be non-NULL and distinct");
    return TPP_ERR_INVALID_ARG;
  }
  if (prec != TPP_FP64 && prec != TPP_FP32 && prec != TPP_BF16) {
    set_error("prec must be TPP_FP64, TPP_FP32 or TPP_BF16");
    return TPP_ERR_INVALID_ARG;
  }
  if (prec == TPP_FP32 && !(c->features & TPP_FEAT_MIXED)) {
    set_error("TPP_FP32 apply needs a context created with TPP_FEAT_MIXED");
    return TPP_ERR_INVALID_ARG;
  }
  if (prec == TPP_FP64 && (c->features & TPP_FEAT_F32_SHIFTS)) {
    set_error("the context keeps its shifted inverses in FP32 only (TPP_FEAT_F32_SHIFTS): "
              "apply with TPP_FP32");
    return TPP_ERR_INVALID_ARG;
  }
  if (prec == TPP_BF16 && !(c->features & TPP_FEAT_BF16)) {
    set_error("TPP_BF16 apply needs a context created with TPP_FEAT_BF16");
    return TPP_ERR_INVALID_ARG;
  }
  if (!c->factors_built) {
    set_error("tpp_build_factors has not been called");
    return TPP_ERR_INVALID_ARG;
  }
  const tpp_ctx v = call_view(c, nrhs);
  TPP_TRY_CUDA(apply_precond(&v, TPP_PC_KRON, prec, b, x, nullptr,
                             static_cast<cudaStream_t>(stream)), "tpp_apply_inverse");
  return TPP_OK;
}

tpp_status tpp_apply_block_jacobi(const tpp_ctx* c, const double* b, double* x, int32_t nrhs,
                                  void* stream) {
  if (tpp_status r = check_ctx(c)) return r;
  if (tpp_status r = check_nrhs(c, nrhs)) return r;
  if (!b || !x || b == x) {
    set_error("b and x must be non-NULL and distinct");
    return TPP_ERR_INVALID_ARG;
  }
  if (!c->bj_built) {
    set_error("tpp_build_block_jacobi has not been called");
    return TPP_ERR_INVALID_ARG;
  }
  const tpp_ctx v = call_view(c, nrhs);
  TPP_TRY_CUDA(v.sys_full_bj
                   ? launch_full_bj_apply(&v, b, x, nullptr, static_cast<cudaStream_t>(stream))
                   : launch_bj_apply(&v, b, x, nullptr, static_cast<cudaStream_t>(stream)),
               "tpp_apply_block_jacobi");
  return TPP_OK;
}

tpp_status dg_apply_sumfact(const tpp_ctx* c, const double* x, double* y, int32_t nrhs,
                            void* stream) {
  if (tpp_status r = check_ctx(c)) return r;
  if (tpp_status r = check_nrhs(c, nrhs)) return r;
  if (!x || !y || x == y) {
    set_error("x and y must be non-NULL and distinct");
    return TPP_ERR_INVALID_ARG;
  }
  const tpp_ctx v = call_view(c, nrhs);
  TPP_TRY_CUDA(apply_operator(&v, x, y, nullptr, static_cast<cudaStream_t>(stream)),
               "dg_apply_sumfact");
  return TPP_OK;
}

tpp_status dg_apply_sumfact_f32(const tpp_ctx* c, const float* x, float* y, int32_t nrhs,
                                void* stream) {
  if (tpp_status r = check_ctx(c)) return r;
  if (tpp_status r = check_nrhs(c, nrhs)) return r;
  if (!x || !y || x == y) {
    set_error("x and y must be non-NULL and distinct");
    return TPP_ERR_INVALID_ARG;
  }
  if (!(c->features & TPP_FEAT_MIXED)) {
    set_error("dg_apply_sumfact_f32 needs TPP_FEAT_MIXED");
    return TPP_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const tpp_ctx v = call_view(c, nrhs);
  float* trf = c->p<float>(c->L.opf) + op_f32_layout(c).tr;
  TPP_TRY_CUDA(launch_traces_f32(&v, x, trf, s, nullptr), "k_traces<float>");
  TPP_TRY_CUDA(launch_dg_apply_f32(&v, x, trf, y, nullptr, s), "k_dg_apply<float>");
  return TPP_OK;
}

tpp_status tpp_apply_inverse_f32(const tpp_ctx* c, const float* b, float* x, int32_t nrhs,
                                 void* stream) {
  if (tpp_status r = check_ctx(c)) return r;
  if (tpp_status r = check_nrhs(c, nrhs)) return r;
  if (!b || !x || b == x) {
    set_error("b and x must be non-NULL and distinct");
    return TPP_ERR_INVALID_ARG;
  }
  if (!(c->features & TPP_FEAT_MIXED) || !c->factors_built) {
    set_error("tpp_apply_inverse_f32 needs TPP_FEAT_MIXED and tpp_build_factors");
    return TPP_ERR_INVALID_ARG;
  }
  const tpp_ctx v = call_view(c, nrhs);
  TPP_TRY_CUDA(launch_apply_f32(&v, b, x, nullptr, static_cast<cudaStream_t>(stream)),
               "tpp_apply_inverse_f32");
  return TPP_OK;
}

tpp_status tpp_get_views(const tpp_ctx* c, tpp_views* o) {
  if (tpp_status r = check_ctx(c)) return r;
  if (!o) {
    set_error("out is NULL");
    return TPP_ERR_INVALID_ARG;
  }
  std::memset(o, 0, sizeof(*o));
  o->sigma = c->p<double>(c->L.sigma);
  o->A1 = c->p<double>(c->L.fA1);
  o->B1 = c->p<double>(c->L.fB1);
  o->A2 = c->p<double>(c->L.fA2);
  o->B2 = c->p<double>(c->L.fB2);
  o->SA = c->p<double>(c->L.fSA);
  o->SB = c->p<double>(c->L.fSB);
  o->Q1 = c->p<double>(c->L.fQ1);
  o->Q2 = two_sided(c) ? c->p<double>(c->L.fQ2) : nullptr;
  o->G = (two_sided(c) || !c->L.fG) ? nullptr : c->p<double>(c->L.fG);
  o->T1 = c->p<double>(c->L.fT1);
  o->T2 = c->p<double>(c->L.fT2);
  o->flags = c->p<int32_t>(c->L.flags);
  o->cond = c->p<double>(c->L.fSC);
  if (c->dim == 3) {
    o->Az = c->p<double>(c->L.fAz);
    o->Azi = c->p<double>(c->L.fAzi);
    o->sigz = c->p<double>(c->L.sigz);
    o->zflags = c->p<int32_t>(c->L.zflags);
  }
  if (c->mu > c->n) {
    o->core = c->p<double>(c->L.kco);
    o->Qb = c->p<double>(c->L.qb);
    o->Rb = c->p<double>(c->L.rb);
    o->qtr = c->p<double>(c->L.qtr);
  }
  if (c->sys_full) {
    o->fA = c->p<double>(c->fb.A);
    o->fB = c->dim == 2 ? c->p<double>(c->fb.B) : nullptr;
    o->fsig = c->p<double>(c->fb.sig);
    o->fflags = c->p<int32_t>(c->fb.flags);
  }
  const Tables* T = c->p<Tables>(c->L.tables);
  o->gl_x = T->x;
  o->gl_w = T->w;
  o->D = T->D;
  return TPP_OK;
}

tpp_status tpp_copy_device(void* dst, const void* src, size_t bytes, void* stream) {
  if (bytes == 0) return TPP_OK;
  if (!dst || !src) {
    set_error("dst and src must be non-NULL");
    return TPP_ERR_INVALID_ARG;
  }
  TPP_TRY_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice,
                               static_cast<cudaStream_t>(stream)), "tpp_copy_device");
  return TPP_OK;
}

tpp_status gmres_solve(tpp_ctx* c, const double* b, double* x, const tpp_gmres_opts* opts,
                       tpp_gmres_result* res, void* stream) {
  if (tpp_status r = check_ctx(c)) return r;
  if (!b || !x || b == x || !opts || !res) {
    set_error("b, x, opts, result must be non-NULL and b != x");
    return TPP_ERR_INVALID_ARG;
  }
  const int m = opts->restart;
  if (m < 1 || m > c->max_restart || opts->max_iters < 1 || !(opts->rtol > 0.0) ||
      opts->pc < TPP_PC_NONE || opts->pc > TPP_PC_BLOCK_JACOBI ||
      (opts->inner_prec != TPP_FP64 && opts->inner_prec != TPP_FP32 &&
       opts->inner_prec != TPP_BF16)) {
    set_error("invalid GMRES options (restart, max_iters, rtol, pc or inner_prec)");
    return TPP_ERR_INVALID_ARG;
  }
  if (opts->pc == TPP_PC_KRON && !c->factors_built) {
    set_error("TPP_PC_KRON needs tpp_build_factors first");
    return TPP_ERR_INVALID_ARG;
  }
  if (opts->pc == TPP_PC_BLOCK_JACOBI && !c->bj_built) {
    set_error("TPP_PC_BLOCK_JACOBI needs tpp_build_block_jacobi first");
    return TPP_ERR_INVALID_ARG;
  }
  if (opts->inner_prec == TPP_BF16 && !(c->features & TPP_FEAT_BF16)) {
    set_error("inner_prec TPP_BF16 needs TPP_FEAT_BF16");
    return TPP_ERR_INVALID_ARG;
  }
  if (opts->pc == TPP_PC_KRON && opts->inner_prec == TPP_FP64 && opts->inner_iters <= 0 &&
      (c->features & TPP_FEAT_F32_SHIFTS)) {
    set_error("TPP_FEAT_F32_SHIFTS: the Kronecker preconditioner runs in FP32 (inner_prec "
              "TPP_FP32, or inner FP32 solves with inner_iters > 0)");
    return TPP_ERR_INVALID_ARG;
  }
  if (opts->inner_prec == TPP_FP32 && !(c->features & TPP_FEAT_MIXED)) {
    set_error("inner_prec TPP_FP32 needs TPP_FEAT_MIXED");
    return TPP_ERR_INVALID_ARG;
  }
  const int kin = opts->inner_iters;
  if (kin < 0 || kin > c->max_restart || (opts->use_graph != 0 && opts->use_graph != 1) ||
      !(opts->inner_rtol >= 0.0)) {
    set_error("inner_iters must be in [0, max_restart], use_graph 0 or 1, inner_rtol >= 0");
    return TPP_ERR_INVALID_ARG;
  }
  if (kin > 0 && (!(c->features & TPP_FEAT_MIXED) || opts->pc != TPP_PC_KRON)) {
    set_error("inner FP32 solves need TPP_FEAT_MIXED and TPP_PC_KRON");
    return TPP_ERR_INVALID_ARG;
  }
  const bool flexible = opts->flexible || opts->inner_prec != TPP_FP64 || kin > 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);   // the capture below swaps it briefly
  const int64_t N = c->N;
  const int nblk = c->partial_blocks, stride = kPartialStride;
  double* V = c->p<double>(c->L.V);
  double* Z = c->p<double>(c->L.Z);
  double* t1 = c->p<double>(c->L.vtmp);
  double* t2 = c->p<double>(c->L.vtmp2);
  double* partials = c->p<double>(c->L.partials);
  GmresState* st = c->p<GmresState>(c->L.gstate);
  const int32_t* done = &st->done;
  const GBuf gb = gbuf_layout(c->max_restart);
  double* gbuf = c->p<double>(c->L.gbuf);
  double *H = gbuf + gb.H, *cs = gbuf + gb.cs, *sn = gbuf + gb.sn, *g = gbuf + gb.g;
  double *h1 = gbuf + gb.h1, *h2 = gbuf + gb.h2, *y = gbuf + gb.y, *invb = gbuf + gb.invb;
  double* scal = gbuf + gb.scal;
  std::memset(res, 0, sizeof(*res));
  // counters of this solve; the reduction tickets start at zero (they are
  // zero after every completed kernel, this also covers an interrupted solve)
  TPP_TRY_CUDA(cudaMemsetAsync(&st->inner_total, 0, sizeof(int32_t), s), "reset inner count");
  TPP_TRY_CUDA(cudaMemsetAsync(st->tickets, 0, sizeof(st->tickets), s), "reset tickets");
  if (c->L.gstate_in) {
    GmresState* sti0 = c->p<GmresState>(c->L.gstate_in);
    TPP_TRY_CUDA(cudaMemsetAsync(sti0->tickets, 0, sizeof(sti0->tickets), s), "reset tickets");
  }
  // inner FP32 solve z = (approximately) S^-1 v for one outer step (mixed mode):
  // GMRES(kin) from 0 on float vectors, the FP32 operator and the FP32
  // Kronecker apply as right preconditioner; every kernel returns at once when
  // the outer cycle is done, and the inner ones also when the inner solve is.
  auto inner_solve = [&](const double* v, double* z) -> tpp_status {
    const GBuf gi = gbuf_layout(c->max_restart);
    double* gb = c->p<double>(c->L.gbuf_in);
    double *Hi = gb + gi.H, *csi = gb + gi.cs, *sni = gb + gi.sn, *g0 = gb + gi.g;
    double *h1i = gb + gi.h1, *h2i = gb + gi.h2, *yi = gb + gi.y, *invbi = gb + gi.invb;
    GmresState* sti = c->p<GmresState>(c->L.gstate_in);
    const int32_t* din = &sti->done;
    float* Vi = c->p<float>(c->L.vi);
    float* tf = c->p<float>(c->L.tf);
    float* trf = c->p<float>(c->L.opf) + op_f32_layout(c).tr;
    TPP_TRY_CUDA(vec_to_float(v, Vi, N, done, s), "inner v0");
    TPP_TRY_CUDA(gmres_cycle_init(sti, g0, 1.0, kin, 1.0, opts->inner_rtol, done, s),
                 "inner init");
    for (int i = 0; i < kin; ++i) {
      float* vi = Vi + (size_t)i * N;
      float* wi = Vi + (size_t)(i + 1) * N;
      TPP_TRY_CUDA(opts->inner_prec == TPP_BF16 ? launch_apply_bf16_f32(c, vi, tf, din, s)
                                                : launch_apply_f32(c, vi, tf, din, s),
                   "inner precond");
      TPP_TRY_CUDA(launch_traces_f32(c, tf, trf, s, din), "inner traces");
      TPP_TRY_CUDA(launch_dg_apply_f32(c, tf, trf, wi, din, s), "inner operator");
      // Gram-Schmidt with selective reorthogonalisation: dots with the basis
      // and ||w||^2 (w is basis vector i + 1), update + norm, then the second
      // pass only when the norm dropped below 1/sqrt 2 of its value
      TPP_TRY_CUDA(gmres_dots<float>(Vi, N, i + 2, wi, partials, stride, nblk, din, h1i,
                                     &sti->tickets[0], s), "inner dots");
      TPP_TRY_CUDA(gmres_update<float>(Vi, N, i + 1, h1i, wi, partials, stride, 2, nblk, din,
                                       nullptr, &sti->tickets[1], sti, Hi, csi, sni, g0, h1i,
                                       h2i, invbi, i, s), "inner update");
      TPP_TRY_CUDA(gmres_dots<float>(Vi, N, i + 1, wi, partials, stride, nblk, &sti->skip_re,
                                     h2i, &sti->tickets[2], s), "inner dots 2");
      TPP_TRY_CUDA(gmres_update<float>(Vi, N, i + 1, h2i, wi, partials, stride, 1, nblk,
                                       &sti->skip_re, nullptr, &sti->tickets[3], sti, Hi, csi, sni,
                                       g0, h1i, h2i, invbi, i, s), "inner norm+givens");
      TPP_TRY_CUDA(vec_scale_f32(wi, wi, N, invbi, 0.0, din, s), "inner scale");
    }
    TPP_TRY_CUDA(gmres_lsq(sti, Hi, g0, yi, s), "inner lsq");
    TPP_TRY_CUDA(gmres_combine_f32(Vi, N, sti, yi, t2, done, s), "inner Vy");
    TPP_TRY_CUDA(accumulate_inner(st, sti, done, s), "inner count");
    TPP_TRY_CUDA(apply_precond(c, TPP_PC_KRON, opts->inner_prec == TPP_BF16 ? TPP_BF16 : TPP_FP32,
                               t2, z, done, s), "inner P^-1");
    return TPP_OK;
  };
  auto read_scalar = [&](const double* dptr, double* hv) -> tpp_status {
    TPP_TRY_CUDA(cudaMemcpyAsync(hv, dptr, sizeof(double), cudaMemcpyDeviceToHost, s), "read");
    TPP_TRY_CUDA(cudaStreamSynchronize(s), "sync");
    return TPP_OK;
  };
  // ||b||
  double bnorm = 0.0;
  TPP_TRY_CUDA(vec_norm(b, N, partials, stride, nblk, scal, s), "norm b");
  if (tpp_status r = read_scalar(scal, &bnorm)) return r;
  if (!std::isfinite(bnorm)) {
    set_error("right-hand side contains NaN or Inf");
    res->status = TPP_ERR_NAN;
    return TPP_ERR_NAN;
  }
  if (bnorm == 0.0) {
    TPP_TRY_CUDA(cudaMemsetAsync(x, 0, (size_t)N * sizeof(double), s), "zero x");
    TPP_TRY_CUDA(cudaStreamSynchronize(s), "sync");
    res->converged = 1;
    res->status = TPP_OK;
    return TPP_OK;
  }
  // r0 = b - A x0 into V[0]
  auto residual = [&](double* beta) -> tpp_status {
    TPP_TRY_CUDA(apply_operator(c, x, t1, nullptr, s), "operator");
    TPP_TRY_CUDA(vec_sub(V, b, t1, N, s), "residual");
    TPP_TRY_CUDA(vec_norm(V, N, partials, stride, nblk, scal, s), "norm r");
    return read_scalar(scal, beta);
  };
  double beta = 0.0;
  if (tpp_status r = residual(&beta)) return r;
  res->true_rel_res = beta / bnorm;
  res->est_rel_res = beta / bnorm;
  int total = 0;
  tpp_status final_status = TPP_ERR_NOT_CONVERGED;
  if (beta <= opts->rtol * bnorm) final_status = TPP_OK;
  while (final_status != TPP_OK && total < opts->max_iters) {
    if (!std::isfinite(beta)) {
      final_status = TPP_ERR_NAN;
      break;
    }
    res->cycles += 1;
    TPP_TRY_CUDA(vec_scale(V, V, N, nullptr, 1.0 / beta, nullptr, s), "scale v0");
    TPP_TRY_CUDA(gmres_cycle_init(st, g, beta, m, bnorm, opts->rtol, nullptr, s), "cycle init");
    // Arnoldi steps are enqueued kLookahead at a time; every kernel of a step
    // returns at once when the device state says the cycle is done (converged,
    // breakdown or restart length reached), so the host reads the state only
    // once per group instead of after every step.
    GmresState hs;
    const int cycle_start = total;
    // one Arnoldi step j (every kernel returns at once when the cycle is done)
    auto step = [&](int j) -> tpp_status {
      double* vj = V + (size_t)j * N;
      double* w = V + (size_t)(j + 1) * N;
      double* z = flexible ? Z + (size_t)j * N : t1;
      if (kin > 0) {
        if (tpp_status r = inner_solve(vj, z)) return r;
      } else {
        TPP_TRY_CUDA(apply_precond(c, opts->pc, opts->inner_prec, vj, z, done, s), "precond");
      }
      TPP_TRY_CUDA(launch_traces(c, z, c->p<double>(c->L.traces), s, done), "traces");
      TPP_TRY_CUDA(launch_dg_apply(c, z, c->p<double>(c->L.traces), w, done, s), "operator");
      // Gram-Schmidt with selective reorthogonalisation (see k_update): the
      // first pass also takes ||w||^2 (w is basis vector j + 1)
      TPP_TRY_CUDA(gmres_dots(V, N, j + 2, w, partials, stride, nblk, done, h1,
                              &st->tickets[0], s), "dots");
      TPP_TRY_CUDA(gmres_update(V, N, j + 1, h1, w, partials, stride, 2, nblk, done, nullptr,
                                &st->tickets[1], st, H, cs, sn, g, h1, h2, invb, j, s),
                   "update");
      TPP_TRY_CUDA(gmres_dots(V, N, j + 1, w, partials, stride, nblk, &st->skip_re, h2,
                              &st->tickets[2], s), "dots 2");
      TPP_TRY_CUDA(gmres_update(V, N, j + 1, h2, w, partials, stride, 1, nblk, &st->skip_re,
                                nullptr, &st->tickets[3], st, H, cs, sn, g, h1, h2, invb, j, s),
                   "norm+givens");
      TPP_TRY_CUDA(vec_scale(w, w, N, invb, 0.0, done, s), "scale");
      return TPP_OK;
    };
    // Arnoldi steps are enqueued in groups of `look`; the host reads the device state
    // once per group.  With use_graph every full group runs as one CUDA graph,
    // captured once per group start and kept in the context (its kernels read only
    // context buffers), so later cycles and solves with the same options replay it.
    const int look = (kin > 0) ? 1 : kLookahead;    // an inner solve is a long step
    if (opts->use_graph) {
      const double key[6] = {(double)m, (double)opts->pc, (double)opts->inner_prec,
                             (double)flexible, (double)kin, opts->inner_rtol};
      if (std::memcmp(key, c->gkey, sizeof(key)) != 0) {
        for (int q = 0; q < kMaxRestart; ++q)
          if (c->gexec[q]) {
            cudaGraphExecDestroy(c->gexec[q]);
            c->gexec[q] = nullptr;
          }
        std::memcpy(c->gkey, key, sizeof(key));
      }
    }
    for (int j0 = 0; j0 < m && total < opts->max_iters; j0 += look) {
      const int j1 = (j0 + look < m) ? j0 + look : m;
      if (opts->use_graph && total + (j1 - j0) <= opts->max_iters) {
        if (!c->gexec[j0]) {
          // captured on the context's own stream (the legacy default stream cannot
          // be captured); capturing runs nothing, the graph is then launched on s
          if (!c->gstream)
            TPP_TRY_CUDA(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking),
                         "capture stream");
          const cudaStream_t user = s;
          s = c->gstream;
          TPP_TRY_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed), "begin capture");
          const int64_t k0 = tpp_kernel_launch_count();
          tpp_status rs = TPP_OK;
          for (int j = j0; j < j1 && rs == TPP_OK; ++j) rs = step(j);
          cudaGraph_t graph = nullptr;
          const cudaError_t ec = cudaStreamEndCapture(s, &graph);
          s = user;
          c->gkernels[j0] = (int32_t)(tpp_kernel_launch_count() - k0);
          count_launch(-c->gkernels[j0]);       // counted per replay instead
          if (rs != TPP_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rs;
          }
          TPP_TRY_CUDA(ec, "end capture");
          const cudaError_t ei = cudaGraphInstantiate(&c->gexec[j0], graph, 0);
          cudaGraphDestroy(graph);
          TPP_TRY_CUDA(ei, "instantiate graph");
        }
        TPP_TRY_CUDA(cudaGraphLaunch(c->gexec[j0], s), "graph launch");
        count_launch(c->gkernels[j0]);
        total += j1 - j0;
      } else {
        for (int j = j0; j < j1 && total < opts->max_iters; ++j) {
          if (tpp_status r = step(j)) return r;
          ++total;
        }
      }
      TPP_TRY_CUDA(cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s), "read state");
      TPP_TRY_CUDA(cudaStreamSynchronize(s), "sync");
      total = cycle_start + hs.k;            // steps the device actually took
      res->est_rel_res = hs.est;
      if (hs.done) break;
    }
    // x += P^-1 (V y) or x += Z y
    TPP_TRY_CUDA(gmres_lsq(st, H, g, y, s), "lsq");
    if (flexible) {
      TPP_TRY_CUDA(gmres_combine(Z, N, st, y, x, 1, s), "x update");
    } else {
      TPP_TRY_CUDA(gmres_combine(V, N, st, y, t2, 0, s), "V y");
      TPP_TRY_CUDA(apply_precond(c, opts->pc, opts->inner_prec, t2, t1, nullptr, s), "precond");
      TPP_TRY_CUDA(vec_axpy(x, t1, 1.0, N, s), "x update");
    }
    if (tpp_status r = residual(&beta)) return r;
    res->true_rel_res = beta / bnorm;
    if (beta <= opts->rtol * bnorm) {
      final_status = TPP_OK;
      break;
    }
    if (hs.breakdown == 2 || !std::isfinite(beta)) {
      final_status = TPP_ERR_NAN;
      break;
    }
  }
  res->iters = total;
  if (kin > 0) {
    int32_t nin = 0;
    TPP_TRY_CUDA(cudaMemcpyAsync(&nin, &st->inner_total, sizeof(nin), cudaMemcpyDeviceToHost, s),
                 "read inner count");
    TPP_TRY_CUDA(cudaStreamSynchronize(s), "sync");
    res->inner_iters = nin;
  }
  res->converged = (final_status == TPP_OK);
  res->status = final_status;
  if (final_status == TPP_ERR_NOT_CONVERGED)
    set_error("GMRES did not reach rtol within max_iters");
  if (final_status == TPP_ERR_NAN) set_error("NaN or Inf in the GMRES residual");
  return final_status;
}

tpp_status tpp_solve_learned(tpp_ctx* c, tpp_mlp* net, double threshold, int32_t iter_limit,
                             const double* b, double* x, const tpp_gmres_opts* opts,
                             tpp_gmres_result* res, tpp_build_report* report, int32_t* rebuilt,
                             void* stream) {
  if (!opts || !res || !rebuilt || iter_limit < 1) {
    set_error("tpp_solve_learned: opts, result, rebuilt non-NULL and iter_limit >= 1");
    return TPP_ERR_INVALID_ARG;
  }
  *rebuilt = 0;
  if (tpp_status r = tpp_build_factors_learned(c, net, threshold, report, stream)) return r;
  tpp_gmres_opts o = *opts;
  o.max_iters = iter_limit < opts->max_iters ? iter_limit : opts->max_iters;
  tpp_status r = gmres_solve(c, b, x, &o, res, stream);
  if (r != TPP_ERR_NOT_CONVERGED || res->converged) return r;
  // iteration threshold exceeded: exact KSVD for every element, continue from x
  const int32_t first = res->iters, first_inner = res->inner_iters, first_cycles = res->cycles;
  *rebuilt = 1;
  tpp_build_report rep2;
  if (tpp_status r2 = tpp_build_factors(c, &rep2, stream)) return r2;
  if (report) {
    report->num_fallback = report->num_elem;
    report->max_cond = rep2.max_cond;
  }
  // the caller's max_iters bounds both solves together
  tpp_gmres_opts o2 = *opts;
  o2.max_iters = opts->max_iters - first;
  if (o2.max_iters < 1) {
    res->status = TPP_ERR_NOT_CONVERGED;
    set_error("GMRES did not reach rtol within max_iters");
    return TPP_ERR_NOT_CONVERGED;
  }
  r = gmres_solve(c, b, x, &o2, res, stream);
  res->iters += first;
  res->inner_iters += first_inner;
  res->cycles += first_cycles;
  return r;
}

}  // extern "C"
