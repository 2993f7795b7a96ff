// Coupled systems of conservation laws (Sec. 5.3 and Sec. 5.6: the Euler equations,
// n_c = dim + 2 components, flux of Eq. euler-flux), linearised around a DG state.
//
// A system context is an ordinary context over E * n_c pseudo-elements (element e,
// component c at e * n_c + c, vectors [E][n_c][n^dim]), isolated from one another,
// whose own coefficients are the "small" diagonal blocks of the Jacobian: component
// c's volume coefficients A_d[c][c] and own-face coefficients 1/2 (A_n[c][c] + lam).
// Factor build, Kronecker apply and block Jacobi act on those small blocks
// unchanged.  The operator (dg_apply_sumfact, gmres_solve) is the coupled one:
//   y_c = M x_c + sum_d sum_c' D_d^T cd[c][c'] x_c'
//         + lifted face fluxes F_c = sum_c' fo[c][c'] u_c'^own + fn[c][c'] u_c'^nbr,
// with the local Lax-Friedrichs flux linearised around the state (lam frozen):
//   fo = dt h^(dim-1) w_t 1/2 (A_n(u0-) + lam I),  fn = dt h^(dim-1) w_t 1/2 (A_n(u0+) - lam I),
//   lam = max(|v- . n| + c-, |v+ . n| + c+),  cd = -dt h^(dim-1) w_q A_d(u0).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tpp_internal.cuh"

namespace tpp {

namespace {

// A_d = dF_d/du of the Euler flux in conserved variables (NC = DIM + 2 components:
// rho, the DIM momenta, rho E), A[d][c][c'] for d < DIM
template <int DIM>
__device__ void euler_jacobians(const double* U, double g, double (*A)[DIM + 2][DIM + 2]) {
  constexpr int NC = DIM + 2, E_ = DIM + 1;
  const double rho = U[0];
  double V[DIM], q2 = 0.0;
  for (int i = 0; i < DIM; ++i) {
    V[i] = U[1 + i] / rho;
    q2 += V[i] * V[i];
  }
  const double g1 = g - 1.0;
  const double p = g1 * (U[E_] - 0.5 * rho * q2);
  const double H = (U[E_] + p) / rho;
  const double phi = 0.5 * g1 * q2;
  for (int d = 0; d < DIM; ++d) {
    const double vd = V[d];
    for (int r = 0; r < NC; ++r)
      for (int c = 0; c < NC; ++c) A[d][r][c] = 0.0;
    A[d][0][1 + d] = 1.0;
    for (int i = 0; i < DIM; ++i) {
      A[d][1 + i][0] = -V[i] * vd + ((i == d) ? phi : 0.0);
      for (int j = 0; j < DIM; ++j)
        A[d][1 + i][1 + j] = ((i == j) ? vd : 0.0) + ((j == d) ? V[i] : 0.0) -
                             ((i == d) ? g1 * V[j] : 0.0);
      A[d][1 + i][E_] = (i == d) ? g1 : 0.0;
    }
    A[d][E_][0] = vd * (phi - H);
    for (int j = 0; j < DIM; ++j) A[d][E_][1 + j] = ((j == d) ? H : 0.0) - g1 * V[j] * vd;
    A[d][E_][E_] = g * vd;
  }
}

// |v . n| + c for the unit normal along axis `ax` (the Cartesian faces)
template <int DIM>
__device__ double euler_speed(const double* U, double g, int ax) {
  const double rho = U[0];
  double q2 = 0.0;
  for (int i = 0; i < DIM; ++i) q2 += (U[1 + i] / rho) * (U[1 + i] / rho);
  const double p = (g - 1.0) * (U[DIM + 1] - 0.5 * rho * q2);
  return fabs(U[1 + ax] / rho) + sqrt(g * p / rho);
}

// volume coefficients at the nodes: sc[d][((e NC + c) NC + c') n^DIM + q] =
// -dt h^(DIM-1) w_q A_d[c][c']; the diagonal entries go to vel (the small blocks'
// "velocity" for the scalar precompute: vel[d][(e NC + c) n^DIM + q] = A_d[c][c])
template <int DIM>
__global__ void k_sys_volume(const Tables* T, int n, int64_t E, double g, double h, double dt,
                             const double* __restrict__ state, double* __restrict__ scx,
                             double* __restrict__ scy, double* __restrict__ scz,
                             double* __restrict__ vel) {
  constexpr int NC = DIM + 2;
  const int nl = (DIM == 2) ? n * n : n * n * n;
  const int64_t tot = E * nl, totp = E * NC * nl;
  const double hf = (DIM == 2) ? h : h * h;
  double* sc[3] = {scx, scy, scz};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / nl;
    const int node = (int)(q % nl), i = node % n, j = (node / n) % n, k = node / (n * n);
    double U[NC], A[DIM][NC][NC];
    for (int c = 0; c < NC; ++c) U[c] = state[(e * NC + c) * nl + node];
    euler_jacobians<DIM>(U, g, A);
    double w = T->w[i] * T->w[j];
    if (DIM == 3) w *= T->w[k];
    const double f = -dt * hf * w;
    for (int d = 0; d < DIM; ++d)
      for (int c = 0; c < NC; ++c) {
        for (int c2 = 0; c2 < NC; ++c2) sc[d][((e * NC + c) * NC + c2) * nl + node] = f * A[d][c][c2];
        vel[d * totp + (e * NC + c) * nl + node] = A[d][c][c];
      }
  }
}

// face coefficients from the state traces tr ([E NC][2 DIM][n^(DIM-1)], k_traces layout)
// and the element neighbours; vfn: the small blocks' own-face coefficient
// 1/2 (A_n[c][c] + lam)
template <int DIM>
__global__ void k_sys_faces(const Tables* T, int n, int64_t E, double g, double h, double dt,
                            const double* __restrict__ tr, const int32_t* __restrict__ nbr,
                            double* __restrict__ sfo, double* __restrict__ sfn,
                            double* __restrict__ vfn) {
  constexpr int NC = DIM + 2, NF = 2 * DIM;
  const int nfl = (DIM == 2) ? n : n * n;
  const int64_t tot = E * NF * nfl;
  const double hf = (DIM == 2) ? h : h * h;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / (NF * nfl);
    const int f = (int)((q / nfl) % NF), t = (int)(q % nfl);
    const int ax = f / 2;
    const double sgn = (f & 1) ? 1.0 : -1.0;           // outward normal sgn e_ax
    const int nb = nbr[e * NF + f];
    double um[NC], up[NC];
    for (int c = 0; c < NC; ++c) {
      um[c] = tr[((e * NC + c) * NF + f) * nfl + t];
      up[c] = (nb >= 0) ? tr[(((int64_t)nb * NC + c) * NF + (f ^ 1)) * nfl + t] : um[c];
    }
    double lam = euler_speed<DIM>(um, g, ax);
    if (nb >= 0) lam = fmax(lam, euler_speed<DIM>(up, g, ax));
    double Am[DIM][NC][NC], Ap[DIM][NC][NC];
    euler_jacobians<DIM>(um, g, Am);
    euler_jacobians<DIM>(up, g, Ap);
    double wt = T->w[t % n];
    if (DIM == 3) wt *= T->w[t / n];
    const double sc = dt * hf * wt;
    for (int c = 0; c < NC; ++c) {
      for (int c2 = 0; c2 < NC; ++c2) {
        const double d = (c == c2) ? lam : 0.0;
        const double jm = sgn * Am[ax][c][c2], jp = sgn * Ap[ax][c][c2];
        const int64_t o = (((e * NF + f) * NC + c) * NC + c2) * nfl + t;
        sfo[o] = sc * 0.5 * (jm + d);
        sfn[o] = (nb >= 0) ? sc * 0.5 * (jp - d) : 0.0;
        if (c == c2) vfn[((e * NC + c) * NF + f) * nfl + t] = 0.5 * (jm + lam);
      }
    }
  }
}

// y = (mass M + dt A) x for the coupled 2D system, one physical element per CTA
__global__ void k_sys_apply_2d(const Tables* T, int n, double hd, const double* __restrict__ scx,
                               const double* __restrict__ scy, const double* __restrict__ sfo,
                               const double* __restrict__ sfn, const int32_t* __restrict__ nbr,
                               const double* __restrict__ x, const double* __restrict__ tr,
                               double* __restrict__ y, const int32_t* skip) {
  constexpr int kNc = 4;
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

// the same for the coupled 3D system (5 components), as k_dg_apply_3d per component
__global__ void k_sys_apply_3d(const Tables* T, int n, double hd, const double* __restrict__ scx,
                               const double* __restrict__ scy, const double* __restrict__ scz,
                               const double* __restrict__ sfo, const double* __restrict__ sfn,
                               const int32_t* __restrict__ nbr, const double* __restrict__ x,
                               const double* __restrict__ tr, double* __restrict__ y,
                               const int32_t* skip) {
  constexpr int kNc = 5;
  if (skip && *skip) return;
  extern __shared__ __align__(16) double sms[];
  const int nn = n * n, n3 = nn * n, tid = threadIdx.x, nt = blockDim.x;
  double* Ds = sms;                 // n^2
  double* wl = Ds + nn;             // w, l0, l1
  double* xs = wl + 3 * n;          // kNc n^3
  double* px = xs + kNc * n3;       // n^3 each
  double* py = px + n3;
  double* pz = py + n3;
  double* fl = pz + n3;             // 6 n^2
  const int64_t e = blockIdx.x;
  for (int q = tid; q < nn; q += nt) Ds[q] = T->D[q];
  for (int q = tid; q < n; q += nt) {
    wl[q] = T->w[q];
    wl[n + q] = T->l0[q];
    wl[2 * n + q] = T->l1[q];
  }
  for (int q = tid; q < kNc * n3; q += nt) xs[q] = x[e * kNc * n3 + q];
  int nbf[6];
  for (int f = 0; f < 6; ++f) nbf[f] = nbr[e * 6 + f];
  __syncthreads();
  for (int c = 0; c < kNc; ++c) {
    for (int q = tid; q < n3; q += nt) {
      double a = 0.0, b = 0.0, d = 0.0;
      for (int c2 = 0; c2 < kNc; ++c2) {
        const int64_t o = ((e * kNc + c) * kNc + c2) * n3 + q;
        const double xv = xs[c2 * n3 + q];
        a += scx[o] * xv;
        b += scy[o] * xv;
        d += scz[o] * xv;
      }
      px[q] = a;
      py[q] = b;
      pz[q] = d;
    }
    for (int q = tid; q < 6 * nn; q += nt) {
      const int f = q / nn, t = q % nn;
      const int nb = nbf[f];
      double F = 0.0;
      for (int c2 = 0; c2 < kNc; ++c2) {
        const int64_t o = (((e * 6 + f) * kNc + c) * kNc + c2) * nn + t;
        F += sfo[o] * tr[((e * kNc + c2) * 6 + f) * nn + t];
        if (nb >= 0) F += sfn[o] * tr[(((int64_t)nb * kNc + c2) * 6 + (f ^ 1)) * nn + t];
      }
      fl[q] = F;
    }
    __syncthreads();
    for (int q = tid; q < n3; q += nt) {
      const int i = q % n, j = (q / n) % n, k = q / nn;
      double acc = hd * wl[i] * wl[j] * wl[k] * xs[c * n3 + q];
      for (int a = 0; a < n; ++a) acc += Ds[a * n + i] * px[a + n * j + nn * k];
      for (int b = 0; b < n; ++b) acc += Ds[b * n + j] * py[i + n * b + nn * k];
      for (int cc = 0; cc < n; ++cc) acc += Ds[cc * n + k] * pz[i + n * j + nn * cc];
      const int qx = j + n * k, qy = i + n * k, qz = i + n * j;
      acc += wl[n + i] * fl[0 * nn + qx] + wl[2 * n + i] * fl[1 * nn + qx];
      acc += wl[n + j] * fl[2 * nn + qy] + wl[2 * n + j] * fl[3 * nn + qy];
      acc += wl[n + k] * fl[4 * nn + qz] + wl[2 * n + k] * fl[5 * nn + qz];
      y[(e * kNc + c) * n3 + q] = acc;
    }
    __syncthreads();
  }
}

// the same operator with all five components in one pass (n <= 8: the 15 n^3 flux
// partials and 30 n^2 face fluxes of an element fit in shared memory), two barriers
// instead of two per component, so every component's coefficient loads are in flight at once
__global__ void k_sys_apply_3d_all(const Tables* T, int n, double hd, const double* __restrict__ scx,
                                   const double* __restrict__ scy, const double* __restrict__ scz,
                                   const double* __restrict__ sfo, const double* __restrict__ sfn,
                                   const int32_t* __restrict__ nbr, const double* __restrict__ x,
                                   const double* __restrict__ tr, double* __restrict__ y,
                                   const int32_t* skip) {
  constexpr int kNc = 5;
  if (skip && *skip) return;
  extern __shared__ __align__(16) double sms[];
  const int nn = n * n, n3 = nn * n, tid = threadIdx.x, nt = blockDim.x;
  double* Ds = sms;                 // n^2
  double* wl = Ds + nn;             // w, l0, l1
  double* xs = wl + 3 * n;          // kNc n^3
  double* pp = xs + kNc * n3;       // [c][d][n^3], d = x, y, z
  double* fl = pp + 3 * kNc * n3;   // [c][6][n^2]
  const int64_t e = blockIdx.x;
  for (int q = tid; q < nn; q += nt) Ds[q] = T->D[q];
  for (int q = tid; q < n; q += nt) {
    wl[q] = T->w[q];
    wl[n + q] = T->l0[q];
    wl[2 * n + q] = T->l1[q];
  }
  for (int q = tid; q < kNc * n3; q += nt) xs[q] = x[e * kNc * n3 + q];
  int nbf[6];
  for (int f = 0; f < 6; ++f) nbf[f] = nbr[e * 6 + f];
  __syncthreads();
  for (int q = tid; q < kNc * n3; q += nt) {
    const int c = q / n3, node = q % n3;
    double a = 0.0, b = 0.0, d = 0.0;
    for (int c2 = 0; c2 < kNc; ++c2) {
      const int64_t o = ((e * kNc + c) * kNc + c2) * n3 + node;
      const double xv = xs[c2 * n3 + node];
      a += scx[o] * xv;
      b += scy[o] * xv;
      d += scz[o] * xv;
    }
    pp[(c * 3 + 0) * n3 + node] = a;
    pp[(c * 3 + 1) * n3 + node] = b;
    pp[(c * 3 + 2) * n3 + node] = d;
  }
  for (int g = tid; g < kNc * 6 * nn; g += nt) {
    const int c = g / (6 * nn), f = (g / nn) % 6, t = g % nn;
    const int nb = nbf[f];
    double F = 0.0;
    for (int c2 = 0; c2 < kNc; ++c2) {
      const int64_t o = (((e * 6 + f) * kNc + c) * kNc + c2) * nn + t;
      F += sfo[o] * tr[((e * kNc + c2) * 6 + f) * nn + t];
      if (nb >= 0) F += sfn[o] * tr[(((int64_t)nb * kNc + c2) * 6 + (f ^ 1)) * nn + t];
    }
    fl[g] = F;
  }
  __syncthreads();
  for (int q = tid; q < kNc * n3; q += nt) {
    const int c = q / n3, node = q % n3;
    const int i = node % n, j = (node / n) % n, k = node / nn;
    const double* px = pp + (c * 3 + 0) * n3;
    const double* py = pp + (c * 3 + 1) * n3;
    const double* pz = pp + (c * 3 + 2) * n3;
    const double* fc = fl + c * 6 * nn;
    double acc = hd * wl[i] * wl[j] * wl[k] * xs[c * n3 + node];
    for (int a = 0; a < n; ++a) acc += Ds[a * n + i] * px[a + n * j + nn * k];
    for (int b = 0; b < n; ++b) acc += Ds[b * n + j] * py[i + n * b + nn * k];
    for (int cc = 0; cc < n; ++cc) acc += Ds[cc * n + k] * pz[i + n * j + nn * cc];
    const int qx = j + n * k, qy = i + n * k, qz = i + n * j;
    acc += wl[n + i] * fc[0 * nn + qx] + wl[2 * n + i] * fc[1 * nn + qx];
    acc += wl[n + j] * fc[2 * nn + qy] + wl[2 * n + j] * fc[3 * nn + qy];
    acc += wl[n + k] * fc[4 * nn + qz] + wl[2 * n + k] * fc[5 * nn + qz];
    y[(e * kNc + c) * n3 + q % n3] = acc;
  }
}

struct SysLayout {
  size_t cx, cy, cz, fo, fn, nbr, total;
};

// NC = dim + 2 components; coupling arrays of the coupled operator after the scalar layout
SysLayout sys_layout(size_t base, int dim, int n, int64_t E) {
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t nc = (size_t)dim + 2, nl = (dim == 2) ? (size_t)n * n : (size_t)n * n * n;
  const size_t nfl = (dim == 2) ? (size_t)n : (size_t)n * n;
  const size_t vol = (size_t)E * nc * nc * nl * 8, fac = (size_t)E * 2 * dim * nc * nc * nfl * 8;
  SysLayout L;
  size_t o = al(base);
  L.cx = o; o += al(vol);
  L.cy = o; o += al(vol);
  L.cz = o; o += (dim == 3) ? al(vol) : 0;
  L.fo = o; o += al(fac);
  L.fn = o; o += al(fac);
  L.nbr = o; o += al((size_t)E * 2 * dim * 4);
  L.total = o;
  return L;
}

const char* sys_validate(const tpp_sys_problem* p, int32_t max_restart, uint32_t features) {
  if (!p) return "tpp_sys_problem is NULL";
  if (p->dim != 2 && p->dim != 3) return "dim must be 2 or 3";
  if (p->flux != TPP_FLUX_EULER || p->nc != p->dim + 2)
    return "flux TPP_FLUX_EULER needs nc = dim + 2 (4 in 2D, 5 in 3D)";
  if (p->n < 1 || p->n > (p->dim == 2 ? TPP_MAX_N : 12))
    return "n must be in 1..32 (2D) or 1..12 (3D)";
  if (p->num_elem < 1 || p->num_elem > (int64_t)1 << 28) return "num_elem out of range";
  if (!(p->gamma > 1.0) || !(p->h > 0.0) || !(p->dt >= 0.0)) return "gamma > 1, h > 0, dt >= 0";
  if (!p->state || !p->nbr) return "state and nbr must be non-NULL";
  // the diagonal 'velocity' scratch (dim + 2 dim / n solution sizes) lives in the Krylov basis
  if ((int64_t)(max_restart + 1) * p->n < (int64_t)p->dim * p->n + 2 * p->dim || max_restart < 5)
    return "system contexts need max_restart >= 5 (and (max_restart + 1) n >= dim (n + 2))";
  if (features & (TPP_FEAT_MIXED | TPP_FEAT_TIME | TPP_FEAT_LEARNED))
    return "system contexts support TPP_FEAT_TWO_SIDED, TPP_FEAT_BLOCK_JACOBI, TPP_FEAT_BF16 "
           "and TPP_FEAT_FULL_BLOCKS";
  if ((features & TPP_FEAT_FULL_BLOCKS) && p->dim == 2 &&
      (p->n > 16 || (features & (TPP_FEAT_TWO_SIDED | TPP_FEAT_BF16))))
    return "TPP_FEAT_FULL_BLOCKS in 2D: n <= 16, without TPP_FEAT_TWO_SIDED or TPP_FEAT_BF16";
  if ((features & TPP_FEAT_FULL_BLOCKS) && p->dim == 3 &&
      ((features & (TPP_FEAT_TWO_SIDED | TPP_FEAT_BF16)) ||
       ((features & TPP_FEAT_BLOCK_JACOBI) && p->n > 6)))
    return "TPP_FEAT_FULL_BLOCKS in 3D: without TPP_FEAT_TWO_SIDED or TPP_FEAT_BF16, and n <= 6 "
           "with TPP_FEAT_BLOCK_JACOBI";
  return nullptr;
}

// features of the small-block context: the full-block factors and their exact LU live
// after the coupling arrays instead
uint32_t small_features(uint32_t f) {
  if (f & TPP_FEAT_FULL_BLOCKS) f &= ~(TPP_FEAT_FULL_BLOCKS | TPP_FEAT_BLOCK_JACOBI);
  return f;
}

tpp_problem small_problem(const tpp_sys_problem* p, const int32_t* iso_nbr) {
  tpp_problem q;
  std::memset(&q, 0, sizeof(q));
  q.dim = p->dim;
  q.n = p->n;
  q.num_elem = p->num_elem * p->nc;
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
  const int n = c->n, nn = n * n;
  if (c->dim == 2) {
    const size_t smem = (size_t)(nn + 3 * n + 4 * nn + 2 * nn + 4 * n) * 8;
    cudaError_t e = cudaFuncSetAttribute(k_sys_apply_2d,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int threads = std::max(64, ((nn + 31) / 32) * 32);
    k_sys_apply_2d<<<(unsigned)c->sys_E, std::min(threads, 1024), smem, s>>>(
        c->p<Tables>(c->L.tables), n, mass * c->prob.h * c->prob.h, c->p<double>(c->sys_cx),
        c->p<double>(c->sys_cy), c->p<double>(c->sys_fo), c->p<double>(c->sys_fn),
        c->p<int32_t>(c->sys_nbr), x, tr, y, skip);
  } else if (n <= 8) {
    const int n3 = nn * n;
    const size_t smem = (size_t)(nn + 3 * n + 5 * n3 + 15 * n3 + 30 * nn) * 8;
    cudaError_t e = cudaFuncSetAttribute(k_sys_apply_3d_all,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sys_apply_3d_all<<<(unsigned)c->sys_E, 256, smem, s>>>(
        c->p<Tables>(c->L.tables), n, mass * c->prob.h * c->prob.h * c->prob.h,
        c->p<double>(c->sys_cx), c->p<double>(c->sys_cy), c->p<double>(c->sys_cz),
        c->p<double>(c->sys_fo), c->p<double>(c->sys_fn), c->p<int32_t>(c->sys_nbr), x, tr, y,
        skip);
  } else {
    const int n3 = nn * n;
    const size_t smem = (size_t)(nn + 3 * n + 5 * n3 + 3 * n3 + 6 * nn) * 8;
    cudaError_t e = cudaFuncSetAttribute(k_sys_apply_3d,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sys_apply_3d<<<(unsigned)c->sys_E, 256, smem, s>>>(
        c->p<Tables>(c->L.tables), n, mass * c->prob.h * c->prob.h * c->prob.h,
        c->p<double>(c->sys_cx), c->p<double>(c->sys_cy), c->p<double>(c->sys_cz),
        c->p<double>(c->sys_fo), c->p<double>(c->sys_fn), c->p<int32_t>(c->sys_nbr), x, tr, y,
        skip);
  }
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
  std::vector<int32_t> iso((size_t)p->num_elem * p->nc * 2 * p->dim, -1);
  const tpp_problem q = small_problem(p, iso.data());
  const size_t base = tpp_workspace_bytes(&q, max_restart, small_features(features));
  if (base == 0) return 0;
  const size_t tot = sys_layout(base, p->dim, p->n, p->num_elem).total;
  if (!(features & TPP_FEAT_FULL_BLOCKS)) return tot;
  return full_layout(tot, p->dim, p->n, p->num_elem, (features & TPP_FEAT_BLOCK_JACOBI) != 0,
                     nullptr);
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
  const int dim = p->dim, nf = 2 * dim, NC = p->nc;
  const int64_t E = p->num_elem;
  std::vector<int32_t> nb((size_t)E * nf);
  {
    cudaError_t e = cudaMemcpy(nb.data(), p->nbr, nb.size() * 4, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_check(e, "read nbr");
  }
  for (size_t i = 0; i < nb.size(); ++i)
    if (nb[i] < -1 || nb[i] >= E) {
      set_error("nbr entry " + std::to_string(i) + " is outside [-1, num_elem)");
      return TPP_ERR_INVALID_ARG;
    }
  std::vector<int32_t> iso((size_t)E * NC * nf, -1);
  const tpp_problem q = small_problem(p, iso.data());
  const uint32_t sf = small_features(features);
  const bool full = (features & TPP_FEAT_FULL_BLOCKS) != 0;
  const size_t base = tpp_workspace_bytes(&q, max_restart, sf);
  const SysLayout SL = sys_layout(base, dim, p->n, E);
  FullOffsets FO;
  const size_t need =
      full ? full_layout(SL.total, dim, p->n, E, (features & TPP_FEAT_BLOCK_JACOBI) != 0, &FO)
           : SL.total;
  if (base == 0 || ws_bytes < need) {
    set_error("workspace smaller than tpp_sys_workspace_bytes");
    return TPP_ERR_WORKSPACE;
  }
  tpp_ctx* c = nullptr;
  if (tpp_status st = tpp_create(&c, &q, max_restart, sf, workspace, ws_bytes, stream))
    return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n = p->n;
  const int64_t N = c->N;                               // E NC n^dim
  double* vel = c->p<double>(c->L.V);                   // scratch: Krylov basis, unused yet
  double* vfn = vel + (size_t)dim * N;
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
  if (dim == 2) {
    k_sys_volume<2><<<152 * 8, 256, 0, s>>>(T, n, E, p->gamma, p->h, p->dt, p->state,
                                            c->p<double>(SL.cx), c->p<double>(SL.cy), nullptr, vel);
    k_sys_faces<2><<<152 * 4, 256, 0, s>>>(T, n, E, p->gamma, p->h, p->dt, tr,
                                           c->p<int32_t>(SL.nbr), c->p<double>(SL.fo),
                                           c->p<double>(SL.fn), vfn);
  } else {
    k_sys_volume<3><<<152 * 8, 256, 0, s>>>(T, n, E, p->gamma, p->h, p->dt, p->state,
                                            c->p<double>(SL.cx), c->p<double>(SL.cy),
                                            c->p<double>(SL.cz), vel);
    k_sys_faces<3><<<152 * 4, 256, 0, s>>>(T, n, E, p->gamma, p->h, p->dt, tr,
                                           c->p<int32_t>(SL.nbr), c->p<double>(SL.fo),
                                           c->p<double>(SL.fn), vfn);
  }
  count_launch(2);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "system coefficients");
  if (tpp_status st = tpp_set_velocity(c, vel, vfn, p->dt, stream)) {   // the small blocks
    tpp_destroy(c);
    return st;
  }
  c->sys_nc = NC;
  c->sys_E = E;
  c->sys_cx = SL.cx;
  c->sys_cy = SL.cy;
  c->sys_cz = SL.cz;
  c->sys_fo = SL.fo;
  c->sys_fn = SL.fn;
  c->sys_nbr = SL.nbr;
  if (full) {
    c->sys_full = true;
    c->sys_full_bj = (features & TPP_FEAT_BLOCK_JACOBI) != 0;
    c->fb = FO;
    if ((e = launch_full_basis(c, s)) != cudaSuccess) return fail(e, "full-block basis");
  }
  *out = c;
  return TPP_OK;
}
