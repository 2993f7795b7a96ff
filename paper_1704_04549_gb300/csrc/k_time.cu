// Time integration of the semi-discrete DG system M u' = J u (Sec. 3.3, Eq.
// mass-u-r; Sec. 3.4 for the implicit systems).  Backward Euler and Alexander's
// three-stage L-stable DIRK method (Sec. 5.2) solve their stages with the
// KSVD-preconditioned GMRES of this library; the classical explicit RK4 method
// (the paper's explicit comparison) applies J through the operator without its
// mass term and inverts the diagonal collocated mass matrix.
#include <cmath>
#include <cstring>
#include <string>

#include "tpp_internal.cuh"

namespace tpp {

namespace {

// y = s M x (mode 0) or y = s M^-1 x (mode 1), M = h^d w (x) w (x) w, per vector block
__global__ void k_mass(const Tables* T, int n, int dim, double hd, int64_t N,
                       const double* __restrict__ x, double* __restrict__ y, double s, int mode,
                       const double* __restrict__ mq, int R) {
  const int nloc = (dim == 2) ? n * n : n * n * n;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(g % nloc);
    const int i = q % n, j = (q / n) % n, k = q / (n * n);
    double m = hd * T->w[i] * T->w[j];
    if (dim == 3) m *= T->w[k];
    if (mq) m = mq[(g / nloc / R) * nloc + q];      // curved elements: w |J_T| (collocated)
    y[g] = mode == 0 ? s * m * x[g] : s * x[g] / m;
  }
}

// out = a0 x0 + a1 x1 + a2 x2 + a3 x3 (terms with a NULL vector are skipped)
__global__ void k_lincomb(int64_t N, double* __restrict__ out, double a0, const double* x0,
                          double a1, const double* x1, double a2, const double* x2, double a3,
                          const double* x3) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N;
       g += (int64_t)gridDim.x * blockDim.x) {
    double v = a0 * x0[g];
    if (x1) v += a1 * x1[g];
    if (x2) v += a2 * x2[g];
    if (x3) v += a3 * x3[g];
    out[g] = v;
  }
}

__global__ void k_scale(double* __restrict__ v, int64_t count, double f) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < count;
       g += (int64_t)gridDim.x * blockDim.x)
    v[g] *= f;
}

cudaError_t mass(const tpp_ctx* c, const double* x, double* y, double s, int mode,
                 cudaStream_t st) {
  const double hd = (c->dim == 2) ? c->prob.h * c->prob.h : c->prob.h * c->prob.h * c->prob.h;
  k_mass<<<152 * 4, 256, 0, st>>>(c->p<Tables>(c->L.tables), c->n, c->dim, hd, c->N, x, y, s,
                                  mode, c->curved ? c->p<double>(c->L.mq) : nullptr, c->R);
  count_launch();
  return cudaGetLastError();
}

cudaError_t lincomb(const tpp_ctx* c, double* out, double a0, const double* x0, double a1 = 0.0,
                    const double* x1 = nullptr, double a2 = 0.0, const double* x2 = nullptr,
                    double a3 = 0.0, const double* x3 = nullptr, cudaStream_t st = nullptr) {
  k_lincomb<<<152 * 4, 256, 0, st>>>(c->N, out, a0, x0, a1, x1, a2, x2, a3, x3);
  count_launch();
  return cudaGetLastError();
}

// operator coefficients (cx, cy, cz, fa: all linear in dt) scaled from the context's
// dt to dt_new; the FP32 copies follow
cudaError_t rescale_dt(tpp_ctx* c, double dt_new, cudaStream_t st) {
  const double f = dt_new / c->prob.dt;
  const int64_t nv = c->E * c->nq;                  // coefficients at the quadrature points
  const int64_t nf = c->E * 2 * c->dim * c->nfq;
  const size_t offs[3] = {c->L.cx, c->L.cy, c->L.cz};
  for (int d = 0; d < c->dim; ++d) {
    k_scale<<<152 * 4, 256, 0, st>>>(c->p<double>(offs[d]), nv, f);
    count_launch();
  }
  k_scale<<<152 * 4, 256, 0, st>>>(c->p<double>(c->L.fa), nf, f);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && (c->features & TPP_FEAT_MIXED)) e = launch_op_to_f32(c, st);
  c->prob.dt = dt_new;
  c->factors_built = false;
  c->bj_built = false;
  return e;
}

// Alexander's three-stage, third-order, L-stable DIRK: gamma the root in (1/6, 1/2) of
// gamma^3 - 3 gamma^2 + 3/2 gamma - 1/6 = 0, tau = (1 + gamma) / 2,
// b1 = -(6 gamma^2 - 16 gamma + 1) / 4, b2 = (6 gamma^2 - 20 gamma + 5) / 4,
// A = [[gamma], [tau - gamma, gamma], [b1, b2, gamma]].
struct Dirk3 {
  double g, A[3][3];
  Dirk3() {
    double x = 0.4358;                       // Newton on the cubic from inside the interval
    for (int it = 0; it < 50; ++it) {
      const double f = ((x - 3.0) * x + 1.5) * x - 1.0 / 6.0;
      const double df = (3.0 * x - 6.0) * x + 1.5;
      const double dx = f / df;
      x -= dx;
      if (std::fabs(dx) <= 1e-17) break;
    }
    g = x;
    const double tau = 0.5 * (1.0 + g);
    const double b1 = -(6.0 * g * g - 16.0 * g + 1.0) / 4.0;
    const double b2 = (6.0 * g * g - 20.0 * g + 5.0) / 4.0;
    std::memset(A, 0, sizeof(A));
    A[0][0] = g;
    A[1][0] = tau - g;
    A[1][1] = g;
    A[2][0] = b1;
    A[2][1] = b2;
    A[2][2] = g;
  }
};

}  // namespace
}  // namespace tpp

using namespace tpp;

extern "C" tpp_status tpp_time_integrate(tpp_ctx* c, double* u, int32_t scheme, double dt,
                                         int32_t steps, int32_t rebuild_each_step,
                                         const tpp_gmres_opts* opts, tpp_time_report* report,
                                         void* stream) {
  if (!c || !u) {
    set_error("tpp_time_integrate: context and u must be non-NULL");
    return TPP_ERR_INVALID_ARG;
  }
  if (!(c->features & TPP_FEAT_TIME)) {
    set_error("tpp_time_integrate needs a context created with TPP_FEAT_TIME");
    return TPP_ERR_INVALID_ARG;
  }
  if (!(dt > 0.0) || !std::isfinite(dt) || steps < 0 || scheme < TPP_TS_BACKWARD_EULER ||
      scheme > TPP_TS_RK4) {
    set_error("tpp_time_integrate: dt > 0 and finite, steps >= 0, a known scheme");
    return TPP_ERR_INVALID_ARG;
  }
  const bool implicit = scheme != TPP_TS_RK4;
  if (implicit && !opts) {
    set_error("tpp_time_integrate: implicit schemes need GMRES options");
    return TPP_ERR_INVALID_ARG;
  }
  if (!(c->prob.dt > 0.0)) {
    set_error("tpp_time_integrate: the context's operator needs dt > 0 (its flux Jacobians "
              "are stored scaled by dt)");
    return TPP_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tpp_time_report rep;
  std::memset(&rep, 0, sizeof(rep));
  const Dirk3 dk;
  const int64_t N = c->N;
  double* tv = c->p<double>(c->L.tvec);
  double *rhs = tv, *U = tv + N, *k0 = tv + 2 * N, *k1 = tv + 3 * N, *k2 = tv + 4 * N,
         *uh = tv + 5 * N;
  double* ks[3] = {k0, k1, k2};
  auto cuda = [&](cudaError_t e, const char* what) { return cuda_check(e, what); };
  auto build = [&]() -> tpp_status {
    tpp_build_report br;
    const tpp_status r = tpp_build_factors(c, &br, stream);
    rep.builds += 1;
    return r;
  };
  // one implicit stage: S U = M uh from the initial guess U = uh
  auto stage = [&]() -> tpp_status {
    if (tpp_status r = cuda(mass(c, uh, rhs, 1.0, 0, s), "mass")) return r;
    if (tpp_status r = cuda(cudaMemcpyAsync(U, uh, (size_t)N * 8, cudaMemcpyDeviceToDevice, s),
                            "copy")) return r;
    tpp_gmres_result res;
    const tpp_status r = gmres_solve(c, rhs, U, opts, &res, stream);
    rep.solves += 1;
    rep.gmres_iters += res.iters;
    if (res.true_rel_res > rep.max_true_rel_res) rep.max_true_rel_res = res.true_rel_res;
    return r;
  };
  tpp_status st = TPP_OK;
  if (implicit) {
    const double target = (scheme == TPP_TS_DIRK3 ? dk.g : 1.0) * dt;
    if (std::fabs(c->prob.dt - target) > 1e-14 * target)
      if ((st = cuda(rescale_dt(c, target, s), "rescale dt"))) return st;
    if (!rebuild_each_step && !c->factors_built && (st = build())) return st;
  }
  for (int step = 0; step < steps && st == TPP_OK; ++step) {
    if (scheme == TPP_TS_BACKWARD_EULER) {
      if (rebuild_each_step && (st = build())) break;
      if ((st = cuda(cudaMemcpyAsync(uh, u, (size_t)N * 8, cudaMemcpyDeviceToDevice, s), "copy")))
        break;
      if ((st = stage())) break;
      if ((st = cuda(cudaMemcpyAsync(u, U, (size_t)N * 8, cudaMemcpyDeviceToDevice, s), "copy")))
        break;
    } else if (scheme == TPP_TS_DIRK3) {
      if (rebuild_each_step && (st = build())) break;
      for (int i = 0; i < 3 && st == TPP_OK; ++i) {
        // uh = u + dt sum_{j<i} a_ij k_j; U solves (M - gamma dt J) U = M uh; k_i = (U - uh) / (gamma dt)
        st = cuda(lincomb(c, uh, 1.0, u, dt * dk.A[i][0], i > 0 ? k0 : nullptr, dt * dk.A[i][1],
                          i > 1 ? k1 : nullptr, 0.0, nullptr, s), "stage input");
        if (st == TPP_OK) st = stage();
        if (st == TPP_OK)
          st = cuda(lincomb(c, ks[i], 1.0 / (dk.g * dt), U, -1.0 / (dk.g * dt), uh, 0.0, nullptr,
                            0.0, nullptr, s), "stage derivative");
      }
      if (st == TPP_OK)   // stiffly accurate: u^{n+1} = U_3
        st = cuda(cudaMemcpyAsync(u, U, (size_t)N * 8, cudaMemcpyDeviceToDevice, s), "copy");
    } else {
      // RK4: f(v) = M^-1 J v = -M^-1 (dt_ctx A v) / dt_ctx
      const double inv = -1.0 / c->prob.dt;
      double* ks4[4] = {k0, k1, k2, rhs};
      const double cst[4] = {0.0, 0.5, 0.5, 1.0};
      for (int i = 0; i < 4 && st == TPP_OK; ++i) {
        const double* v = u;
        if (i > 0) {
          st = cuda(lincomb(c, uh, 1.0, u, cst[i] * dt, ks4[i - 1], 0.0, nullptr, 0.0, nullptr, s),
                    "stage input");
          v = uh;
        }
        if (st == TPP_OK) st = cuda(launch_traces(c, v, c->p<double>(c->L.traces), s), "traces");
        if (st == TPP_OK)
          st = cuda(launch_dg_apply_flux(c, v, c->p<double>(c->L.traces), U, s), "flux");
        if (st == TPP_OK) st = cuda(mass(c, U, ks4[i], inv, 1, s), "mass inverse");
      }
      if (st == TPP_OK)
        st = cuda(lincomb(c, u, 1.0, u, dt / 6.0, k0, dt / 3.0, k1, dt / 3.0, k2, s), "update");
      if (st == TPP_OK)
        st = cuda(lincomb(c, u, 1.0, u, dt / 6.0, rhs, 0.0, nullptr, 0.0, nullptr, s), "update");
    }
    if (st == TPP_OK) rep.steps += 1;
  }
  if (st == TPP_OK) st = cuda(cudaStreamSynchronize(s), "tpp_time_integrate sync");
  if (report) *report = rep;
  return st;
}
