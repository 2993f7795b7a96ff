// Coupled systems of conservation laws (Sec. 5.3 and Sec. 5.6: the Euler equations,
// n_c = 4 components in 2D, flux of Eq. euler-flux), linearised around a DG state.
//
// A system context is an ordinary context over E * n_c pseudo-elements (element e,
// component c at e * n_c + c, vectors [E][n_c][n^2]), isolated from one another,
// whose own coefficients are the "small" diagonal blocks of the Jacobian: component
// c's volume coefficients A_d[c][c] and own-face coefficients 1/2 (A_n[c][c] + lam).
// Factor build, Kronecker apply and block Jacobi act on those small blocks
// unchanged.  The operator (dg_apply_sumfact, gmres_solve) is the coupled one:
//   y_c = M x_c + sum_c' [ sum_k D_ki cx[c][c'] x_c' + sum_l D_lj cy[c][c'] x_c' ]
//         + lifted face fluxes F_c = sum_c' fo[c][c'] u_c'^own + fn[c][c'] u_c'^nbr,
// with the local Lax-Friedrichs flux linearised around the state (lam frozen):
//   fo = dt h w_t 1/2 (A_n(u0-) + lam I),  fn = dt h w_t 1/2 (A_n(u0+) - lam I),
//   lam = max(|v- . n| + c-, |v+ . n| + c+),  cx = -dt h w_i w_j A_x(u0), cy likewise.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tpp_internal.cuh"

namespace tpp {

namespace {

constexpr int kNc = 4;

// A_x, A_y = dF/du of Eq. euler-flux in conserved variables, |v.n| + c for normal nv
__device__ void euler_jacobians(const double U[kNc], double g, double Ax[kNc][kNc],
                                double Ay[kNc][kNc]) {
  const double rho = U[0], u = U[1] / rho, v = U[2] / rho;
  const double g1 = g - 1.0;
  const double p = g1 * (U[3] - 0.5 * rho * (u * u + v * v));
  const double H = (U[3] + p) / rho;
  const double phi = 0.5 * g1 * (u * u + v * v);
  Ax[0][0] = 0.0;            Ax[0][1] = 1.0;                Ax[0][2] = 0.0;              Ax[0][3] = 0.0;
  Ax[1][0] = phi - u * u;    Ax[1][1] = (3.0 - g) * u;      Ax[1][2] = -g1 * v;          Ax[1][3] = g1;
  Ax[2][0] = -u * v;         Ax[2][1] = v;                  Ax[2][2] = u;                Ax[2][3] = 0.0;
  Ax[3][0] = u * (phi - H);  Ax[3][1] = H - g1 * u * u;     Ax[3][2] = -g1 * u * v;      Ax[3][3] = g * u;
  Ay[0][0] = 0.0;            Ay[0][1] = 0.0;                Ay[0][2] = 1.0;              Ay[0][3] = 0.0;
  Ay[1][0] = -u * v;         Ay[1][1] = v;                  Ay[1][2] = u;                Ay[1][3] = 0.0;
  Ay[2][0] = phi - v * v;    Ay[2][1] = -g1 * u;            Ay[2][2] = (3.0 - g) * v;    Ay[2][3] = g1;
  Ay[3][0] = v * (phi - H);  Ay[3][1] = -g1 * u * v;        Ay[3][2] = H - g1 * v * v;   Ay[3][3] = g * v;
}

__device__ double euler_speed(const double U[kNc], double g, double nx, double ny) {
  const double rho = U[0], u = U[1] / rho, v = U[2] / rho;
  const double p = (g - 1.0) * (U[3] - 0.5 * rho * (u * u + v * v));
  return fabs(u * nx + v * ny) + sqrt(g * p / rho);
}

// volume coefficients at the nodes; the diagonal entries go to vel (the small blocks'
// "velocity" for the scalar precompute: vel[g] = A_x[c][c], vel[Ep n^2 + g] = A_y[c][c])
__global__ void k_sys_volume(const Tables* T, int n, int64_t E, double g, double h, double dt,
                             const double* __restrict__ state, double* __restrict__ scx,
                             double* __restrict__ scy, double* __restrict__ vel) {
  const int nn = n * n;
  const int64_t tot = E * nn, totp = E * kNc * nn;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / nn;
    const int node = (int)(q % nn), i = node % n, j = node / n;
    double U[kNc], Ax[kNc][kNc], Ay[kNc][kNc];
    for (int c = 0; c < kNc; ++c) U[c] = state[(e * kNc + c) * nn + node];
    euler_jacobians(U, g, Ax, Ay);
    const double f = -dt * h * T->w[i] * T->w[j];
    for (int c = 0; c < kNc; ++c) {
      for (int c2 = 0; c2 < kNc; ++c2) {
        const int64_t o = ((e * kNc + c) * kNc + c2) * nn + node;
        scx[o] = f * Ax[c][c2];
        scy[o] = f * Ay[c][c2];
      }
      vel[(e * kNc + c) * nn + node] = Ax[c][c];
      vel[totp + (e * kNc + c) * nn + node] = Ay[c][c];
    }
  }
}

// face coefficients from the state traces tr ([E n_c][4][n], k_traces layout) and the
// element neighbours; vfn: the small blocks' own-face coefficient 1/2 (A_n[c][c] + lam)
__global__ void k_sys_faces(const Tables* T, int n, int64_t E, double g, double h, double dt,
                            const double* __restrict__ tr, const int32_t* __restrict__ nbr,
                            double* __restrict__ sfo, double* __restrict__ sfn,
                            double* __restrict__ vfn) {
  const int64_t tot = E * 4 * n;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / (4 * n);
    const int f = (int)((q / n) % 4), t = (int)(q % n);
    const double nx = (f == 0) ? -1.0 : (f == 1) ? 1.0 : 0.0;
    const double ny = (f == 2) ? -1.0 : (f == 3) ? 1.0 : 0.0;
    const int nb = nbr[e * 4 + f];
    double um[kNc], up[kNc];
    for (int c = 0; c < kNc; ++c) {
      um[c] = tr[((e * kNc + c) * 4 + f) * n + t];
      up[c] = (nb >= 0) ? tr[(((int64_t)nb * kNc + c) * 4 + (f ^ 1)) * n + t] : um[c];
    }
    double lam = euler_speed(um, g, nx, ny);
    if (nb >= 0) lam = fmax(lam, euler_speed(up, g, nx, ny));
    double Ax[kNc][kNc], Ay[kNc][kNc], Bx[kNc][kNc], By[kNc][kNc];
    euler_jacobians(um, g, Ax, Ay);
    euler_jacobians(up, g, Bx, By);
    const double sc = dt * h * T->w[t];
    for (int c = 0; c < kNc; ++c) {
      for (int c2 = 0; c2 < kNc; ++c2) {
        const double d = (c == c2) ? lam : 0.0;
        const double jm = nx * Ax[c][c2] + ny * Ay[c][c2];
        const double jp = nx * Bx[c][c2] + ny * By[c][c2];
        const int64_t o = (((e * 4 + f) * kNc + c) * kNc + c2) * n + t;
        sfo[o] = sc * 0.5 * (jm + d);
        sfn[o] = (nb >= 0) ? sc * 0.5 * (jp - d) : 0.0;
        if (c == c2) vfn[((e * kNc + c) * 4 + f) * n + t] = 0.5 * (jm + lam);
      }
    }
  }
}

// y = (mass M + dt A) x for the coupled system, one physical element per CTA
__global__ void k_sys_apply_2d(const Tables* T, int n, double hd, const double* __restrict__ scx,
                               const double* __restrict__ scy, const double* __restrict__ sfo,
                               const double* __restrict__ sfn, const int32_t* __restrict__ nbr,
                               const double* __restrict__ x, const double* __restrict__ tr,
                               double* __restrict__ y, const int32_t* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) double sms[];
  const int nn = n * n, tid = threadIdx.x, nt = blockDim.x;
  double* Ds = sms;                 // n^2
  double* wl = Ds + nn;             // w, l0, l1
  double* xs = wl + 3 * n;          // kNc n^2
  double* px = xs + kNc * nn;       // n^2
  double* py = px + nn;             // n^2
  double* fl = py + nn;             // 4 n
  const int64_t e = blockIdx.x;
  for (int q = tid; q < nn; q += nt) Ds[q] = T->D[q];
  for (int q = tid; q < n; q += nt) {
    wl[q] = T->w[q];
    wl[n + q] = T->l0[q];
    wl[2 * n + q] = T->l1[q];
  }
  for (int q = tid; q < kNc * nn; q += nt) xs[q] = x[e * kNc * nn + q];
  int nbf[4];
  for (int f = 0; f < 4; ++f) nbf[f] = nbr[e * 4 + f];
  __syncthreads();
  for (int c = 0; c < kNc; ++c) {
    for (int q = tid; q < nn; q += nt) {
      double a = 0.0, b = 0.0;
      for (int c2 = 0; c2 < kNc; ++c2) {
        const int64_t o = ((e * kNc + c) * kNc + c2) * nn + q;
        a += scx[o] * xs[c2 * nn + q];
        b += scy[o] * xs[c2 * nn + q];
      }
      px[q] = a;
      py[q] = b;
    }
    for (int q = tid; q < 4 * n; q += nt) {
      const int f = q / n, t = q % n;
      const int nb = nbf[f];
      double F = 0.0;
      for (int c2 = 0; c2 < kNc; ++c2) {
        const int64_t o = (((e * 4 + f) * kNc + c) * kNc + c2) * n + t;
        F += sfo[o] * tr[((e * kNc + c2) * 4 + f) * n + t];
        if (nb >= 0) F += sfn[o] * tr[(((int64_t)nb * kNc + c2) * 4 + (f ^ 1)) * n + t];
      }
      fl[q] = F;
    }
    __syncthreads();
    for (int q = tid; q < nn; q += nt) {
      const int i = q % n, j = q / n;
      double acc = hd * wl[i] * wl[j] * xs[c * nn + q];
      for (int k = 0; k < n; ++k) acc += Ds[k * n + i] * px[k + n * j];
      for (int l = 0; l < n; ++l) acc += Ds[l * n + j] * py[i + n * l];
      acc += wl[n + i] * fl[j] + wl[2 * n + i] * fl[n + j];
      acc += wl[n + j] * fl[2 * n + i] + wl[2 * n + j] * fl[3 * n + i];
      y[(e * kNc + c) * nn + q] = acc;
    }
    __syncthreads();
  }
}

struct SysLayout {
  size_t cx, cy, fo, fn, nbr, total;
};

SysLayout sys_layout(size_t base, int n, int64_t E) {
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t vol = (size_t)E * kNc * kNc * n * n * 8, fac = (size_t)E * 4 * kNc * kNc * n * 8;
  SysLayout L;
  size_t o = al(base);
  L.cx = o; o += al(vol);
  L.cy = o; o += al(vol);
  L.fo = o; o += al(fac);
  L.fn = o; o += al(fac);
  L.nbr = o; o += al((size_t)E * 4 * 4);
  L.total = o;
  return L;
}

const char* sys_validate(const tpp_sys_problem* p, int32_t max_restart, uint32_t features) {
  if (!p) return "tpp_sys_problem is NULL";
  if (p->dim != 2) return "systems are implemented in 2D";
  if (p->flux != TPP_FLUX_EULER || p->nc != kNc) return "flux TPP_FLUX_EULER needs nc = 4";
  if (p->n < 1 || p->n > TPP_MAX_N) return "n must be in 1..32";
  if (p->num_elem < 1 || p->num_elem > (int64_t)1 << 28) return "num_elem out of range";
  if (!(p->gamma > 1.0) || !(p->h > 0.0) || !(p->dt >= 0.0)) return "gamma > 1, h > 0, dt >= 0";
  if (!p->state || !p->nbr) return "state and nbr must be non-NULL";
  if (max_restart < 5) return "system contexts need max_restart >= 5";
  if (features & (TPP_FEAT_MIXED | TPP_FEAT_TIME | TPP_FEAT_LEARNED))
    return "system contexts support TPP_FEAT_TWO_SIDED, TPP_FEAT_BLOCK_JACOBI and TPP_FEAT_BF16";
  return nullptr;
}

tpp_problem small_problem(const tpp_sys_problem* p, const int32_t* iso_nbr) {
  tpp_problem q;
  std::memset(&q, 0, sizeof(q));
  q.dim = 2;
  q.n = p->n;
  q.num_elem = p->num_elem * kNc;
  q.nrhs = 1;
  q.mu = 0;
  q.h = p->h;
  q.dt = p->dt;
  q.nbr = iso_nbr;
  return q;
}

}  // namespace

cudaError_t launch_sys_apply(const tpp_ctx* c, const double* x, const double* tr, double* y,
                             const int32_t* skip, cudaStream_t s, double mass) {
  const int n = c->n;
  const size_t smem = (size_t)(n * n + 3 * n + kNc * n * n + 2 * n * n + 4 * n) * 8;
  cudaError_t e = cudaFuncSetAttribute(k_sys_apply_2d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int threads = std::max(64, ((n * n + 31) / 32) * 32);
  k_sys_apply_2d<<<(unsigned)c->sys_E, std::min(threads, 1024), smem, s>>>(
      c->p<Tables>(c->L.tables), n, mass * c->prob.h * c->prob.h, c->p<double>(c->sys_cx),
      c->p<double>(c->sys_cy), c->p<double>(c->sys_fo), c->p<double>(c->sys_fn),
      c->p<int32_t>(c->sys_nbr), x, tr, y, skip);
  count_launch();
  return cudaGetLastError();
}

}  // namespace tpp

using namespace tpp;

extern "C" size_t tpp_sys_workspace_bytes(const tpp_sys_problem* p, int32_t max_restart,
                                          uint32_t features) {
  if (const char* why = sys_validate(p, max_restart, features)) {
    set_error(why);
    return 0;
  }
  std::vector<int32_t> iso((size_t)p->num_elem * kNc * 4, -1);
  const tpp_problem q = small_problem(p, iso.data());
  const size_t base = tpp_workspace_bytes(&q, max_restart, features);
  if (base == 0) return 0;
  return sys_layout(base, p->n, p->num_elem).total;
}

extern "C" tpp_status tpp_create_system(tpp_ctx** out, const tpp_sys_problem* p,
                                        int32_t max_restart, uint32_t features, void* workspace,
                                        size_t ws_bytes, void* stream) {
  if (!out) {
    set_error("out is NULL");
    return TPP_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (const char* why = sys_validate(p, max_restart, features)) {
    set_error(why);
    return TPP_ERR_INVALID_ARG;
  }
  const int64_t E = p->num_elem;
  std::vector<int32_t> nb((size_t)E * 4);
  {
    cudaError_t e = cudaMemcpy(nb.data(), p->nbr, nb.size() * 4, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_check(e, "read nbr");
  }
  for (size_t i = 0; i < nb.size(); ++i)
    if (nb[i] < -1 || nb[i] >= E) {
      set_error("nbr entry " + std::to_string(i) + " is outside [-1, num_elem)");
      return TPP_ERR_INVALID_ARG;
    }
  std::vector<int32_t> iso((size_t)E * kNc * 4, -1);
  const tpp_problem q = small_problem(p, iso.data());
  const size_t base = tpp_workspace_bytes(&q, max_restart, features);
  const SysLayout SL = sys_layout(base, p->n, E);
  if (base == 0 || ws_bytes < SL.total) {
    set_error("workspace smaller than tpp_sys_workspace_bytes");
    return TPP_ERR_WORKSPACE;
  }
  tpp_ctx* c = nullptr;
  if (tpp_status st = tpp_create(&c, &q, max_restart, features, workspace, ws_bytes, stream))
    return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n = p->n;
  const int64_t Ep = E * kNc, N = Ep * n * n;
  double* vel = c->p<double>(c->L.V);                    // scratch: Krylov basis, unused yet
  double* vfn = vel + 2 * N;
  auto fail = [&](cudaError_t e, const char* what) {
    const tpp_status st = cuda_check(e, what);
    tpp_destroy(c);
    return st;
  };
  cudaError_t e = cudaMemcpyAsync(c->ws + SL.nbr, nb.data(), nb.size() * 4,
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(e, "copy nbr");
  double* tr = c->p<double>(c->L.traces);
  if ((e = launch_traces(c, p->state, tr, s)) != cudaSuccess) return fail(e, "state traces");
  const Tables* T = c->p<Tables>(c->L.tables);
  k_sys_volume<<<152 * 8, 256, 0, s>>>(T, n, E, p->gamma, p->h, p->dt, p->state,
                                       c->p<double>(SL.cx), c->p<double>(SL.cy), vel);
  count_launch();
  k_sys_faces<<<152 * 4, 256, 0, s>>>(T, n, E, p->gamma, p->h, p->dt, tr,
                                      c->p<int32_t>(SL.nbr), c->p<double>(SL.fo),
                                      c->p<double>(SL.fn), vfn);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "system coefficients");
  if (tpp_status st = tpp_set_velocity(c, vel, vfn, p->dt, stream)) {   // the small blocks
    tpp_destroy(c);
    return st;
  }
  c->sys_nc = kNc;
  c->sys_E = E;
  c->sys_cx = SL.cx;
  c->sys_cy = SL.cy;
  c->sys_fo = SL.fo;
  c->sys_fn = SL.fn;
  c->sys_nbr = SL.nbr;
  *out = c;
  return TPP_OK;
}
