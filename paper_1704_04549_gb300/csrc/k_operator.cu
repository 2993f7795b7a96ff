// 1D tables, flux-Jacobian precomputation and the sum-factorised DG operator.
//
// Sec. 3.2 (G, D, W; collocated Gauss-Legendre quadrature so G = I),
// Alg. matrix-free-matvec (steps 1-2 precomputed once, step 3 per matvec),
// Eq. jac-entries (volume and face terms of the Jacobian).
#include "tpp_internal.cuh"

namespace tpp {

// ---------------------------------------------------------------------------
// Gauss-Legendre nodes by Newton's method on the three-term Legendre
// recurrence (initial guesses cos(pi (k + 3/4) / (n + 1/2))), weights
// 2 / ((1 - x^2) P_n'(x)^2); barycentric differentiation matrix
// D_aj = (lambda_j / lambda_a) / (x_a - x_j), D_aa = -sum_{j != a} D_aj
// (Berrut & Trefethen 2004); endpoint values by the barycentric formula.
__global__ void k_tables(Tables* T, int n) {
  __shared__ double lam[TPP_MAX_N];
  const int i = threadIdx.x;
  if (i < n) gauss_legendre_node(n, i, &T->x[i], &T->w[i]);
  __syncthreads();
  if (i < n) {
    double prod = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != i) prod *= (T->x[i] - T->x[m]);
    lam[i] = 1.0 / prod;
  }
  __syncthreads();
  if (i < n) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      const double d = (lam[j] / lam[i]) / (T->x[i] - T->x[j]);
      T->D[i * n + j] = d;
      diag -= d;
    }
    T->D[i * n + i] = diag;
    // phi_i(e) = (lam_i / (e - x_i)) / sum_m lam_m / (e - x_m), e in {0, 1}
    double s0 = 0.0, s1 = 0.0;
    for (int m = 0; m < n; ++m) {
      s0 += lam[m] / (0.0 - T->x[m]);
      s1 += lam[m] / (1.0 - T->x[m]);
    }
    T->l0[i] = (lam[i] / (0.0 - T->x[i])) / s0;
    T->l1[i] = (lam[i] / (1.0 - T->x[i])) / s1;
  }
  __syncthreads();
  if (i < n) {
    T->wf[i] = __double2float_rn(T->w[i]);
    T->l0f[i] = __double2float_rn(T->l0[i]);
    T->l1f[i] = __double2float_rn(T->l1[i]);
    for (int j = 0; j < n; ++j) T->Df[i * n + j] = __double2float_rn(T->D[i * n + j]);
  }
}

cudaError_t launch_tables(const tpp_ctx* c, cudaStream_t s) {
  k_tables<<<1, 32, 0, s>>>(c->p<Tables>(c->L.tables), c->n);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Element-independent basis of the 2D rearranged block.  With collocated
// quadrature every x-term of the diagonal block carries delta_{l j} and every
// y-term delta_{k i}, so (Sec. 4.1 rearrangement, row j + n l, column i + n k)
//     A~ = E (Cx^T Z^T + Dg^T E^T) + Z Cy E^T,
// E selecting the n "diagonal" indices d (n + 1), Cx / Cy per-block
// coefficients, Dg the diagonal of the block (mass and anything else on it),
// and Z (n^2 x (n + 2)) a fixed basis: vec(D^T e_c e_c^T) (c < n),
// vec(l1 l1^T), vec(l0 l0^T).  Householder QR of the off-diagonal rows of Z
// gives Z = E Zd + Qo Rz and A~ = Q M Q^T with Q = [E | Qo] and the small
// core M (only products with A~ are needed; here they collapse onto M).
// One CTA.
__global__ void k_struct_qr(const Tables* T, int n, double* work, double* tau, double* Zd,
                            double* Rz, double* Qo) {
  __shared__ double red[32];
  __shared__ double sh_s[TPP_MAX_N + 2];
  const int nc = n + 2;
  const int Ro = n * n - n;
  const int rz = Ro < nc ? Ro : nc;
  const int tid = threadIdx.x, nt = blockDim.x;
  // Zd[d][c] = Z[d (n+1), c]
  for (int q = tid; q < n * nc; q += nt) {
    const int d = q / nc, cc = q % nc;
    double v;
    if (cc < n) v = (cc == d) ? T->D[d * n + d] : 0.0;
    else if (cc == n) v = T->l1[d] * T->l1[d];
    else v = T->l0[d] * T->l0[d];
    Zd[q] = v;
  }
  // off-diagonal rows: o -> (a, b), a != b, increasing a + n b; column-major work
  for (int q = tid; q < Ro * nc; q += nt) {
    const int cc = q / Ro, o = q % Ro;
    const int b = o / (n - 1), a0 = o % (n - 1), a = a0 + (a0 >= b ? 1 : 0);
    double v;
    if (cc < n) v = (b == cc) ? T->D[cc * n + a] : 0.0;
    else if (cc == n) v = T->l1[a] * T->l1[b];
    else v = T->l0[a] * T->l0[b];
    work[q] = v;
  }
  __syncthreads();
  for (int k = 0; k < rz; ++k) {
    double* col = work + (size_t)k * Ro;
    double part = 0.0;
    for (int o = k + 1 + tid; o < Ro; o += nt) part += col[o] * col[o];
    const double sig = block_sum(part, red);
    const double alpha = col[k];
    double beta = 0.0, t = 0.0, scal = 0.0;
    if (sig > 0.0) {
      beta = -copysign(sqrt(alpha * alpha + sig), alpha);
      t = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    __syncthreads();
    if (sig > 0.0) {
      for (int o = k + 1 + tid; o < Ro; o += nt) col[o] *= scal;   // v = [1, col[k+1:] * scal]
    }
    __syncthreads();
    if (tid == 0) {
      tau[k] = t;
      if (sig > 0.0) col[k] = beta;
    }
    // apply H = I - t v v^T to columns k+1..nc-1 (one warp per column)
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    for (int cc = k + 1 + wid; cc < nc; cc += nw) {
      double* cj = work + (size_t)cc * Ro;
      double sdot = 0.0;
      for (int o = k + lane; o < Ro; o += 32) sdot += (o == k ? 1.0 : col[o]) * cj[o];
      sdot = warp_sum(sdot);
      if (lane == 0) sh_s[cc] = sdot;
    }
    __syncthreads();
    for (int cc = k + 1 + wid; cc < nc; cc += nw) {
      double* cj = work + (size_t)cc * Ro;
      const double f = t * sh_s[cc];
      for (int o = k + lane; o < Ro; o += 32) cj[o] -= f * (o == k ? 1.0 : col[o]);
    }
    __syncthreads();
  }
  // R (rz x nc), row-major
  for (int q = tid; q < rz * nc; q += nt) {
    const int r = q / nc, cc = q % nc;
    Rz[q] = (cc >= r) ? work[(size_t)cc * Ro + r] : 0.0;
  }
  // explicit Qo (Ro x rz), column-major: Q = H_0 ... H_{rz-1} I[:, :rz]
  for (int q = tid; q < Ro * rz; q += nt) {
    const int cc = q / Ro, o = q % Ro;
    Qo[q] = (o == cc) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int k = rz - 1; k >= 0; --k) {
    const double* v = work + (size_t)k * Ro;
    const double t = tau[k];
    for (int cc = k + wid; cc < rz; cc += nw) {
      double* qc = Qo + (size_t)cc * Ro;
      double sdot = 0.0;
      for (int o = k + lane; o < Ro; o += 32) sdot += (o == k ? 1.0 : v[o]) * qc[o];
      sdot = warp_sum(sdot);
      const double f = t * sdot;
      for (int o = k + lane; o < Ro; o += 32) qc[o] -= f * (o == k ? 1.0 : v[o]);
    }
    __syncthreads();
  }
}

cudaError_t launch_struct_qr(const tpp_ctx* c, cudaStream_t s) {
  k_struct_qr<<<1, 1024, 0, s>>>(c->p<Tables>(c->L.tables), c->n, c->p<double>(c->L.qr_work),
                                 c->p<double>(c->L.qr_tau), c->p<double>(c->L.zd),
                                 c->p<double>(c->L.rz), c->p<double>(c->L.qo));
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Flux Jacobians (Alg. matrix-free-matvec step 2).  For advection
// dF_c/du = a_c, and the upwind flux through a face depends on a.n_outward.
// Stored pre-multiplied by the quadrature weights and metric factors:
//   cX[e][i + n j (+ n^2 k)] = -dt h^(d-1) w_i w_j (w_k) a_X(node)     (X = x, y, z)
//   fa[e][f][t]              = dt h^(d-1) (tangential weights) (a.n_outward)(face node)
// from the caller's arrays (NULL: a zero field).
__global__ void k_precompute(const double* __restrict__ wq, int dim, int n, int64_t E, double h,
                             double dt, const double* __restrict__ vel,
                             const double* __restrict__ vfn, double* cx, double* cy, double* cz,
                             double* fa) {
  // n: quadrature points per direction (the nodes, or the mu-point rule), weights wq
  const int nloc = (dim == 2) ? n * n : n * n * n;
  const int nfl = (dim == 2) ? n : n * n;
  const int64_t tot_v = E * nloc, tot_f = E * 2 * dim * nfl;
  const double hf = (dim == 2) ? h : h * h;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < tot_v + tot_f;
       g += (int64_t)gridDim.x * blockDim.x) {
    if (g < tot_v) {
      const int q = (int)(g % nloc);
      const int i = q % n, j = (q / n) % n, k = q / (n * n);
      double wv = wq[i] * wq[j];
      if (dim == 3) wv *= wq[k];
      const double f = -dt * hf * wv;
      cx[g] = vel ? f * vel[g] : 0.0;
      cy[g] = vel ? f * vel[tot_v + g] : 0.0;
      if (dim == 3) cz[g] = vel ? f * vel[2 * tot_v + g] : 0.0;
    } else {
      const int64_t gf = g - tot_v;
      const int q = (int)(gf % nfl);
      const int t0 = q % n, t1 = q / n;   // tangential indices (first tangential fastest)
      const double wt = (dim == 2) ? wq[t0] : wq[t0] * wq[t1];
      fa[gf] = vfn ? dt * hf * wt * vfn[gf] : 0.0;
    }
  }
}

// Curved elements (2D): the caller's metric terms at the quadrature points of the rule
// (n nodes or mu points per direction, weights wq): mq = w |J_T|, cx = -dt w F~_x,
// cy = -dt w F~_y with F~ = |J_T| J_T^-1 a, and fa = dt w_t a . (|J_T| J_T^-T N^).
__global__ void k_metric_2d(const double* __restrict__ wq, int m, int64_t E, double dt,
                            const double* __restrict__ jdet, const double* __restrict__ flux,
                            const double* __restrict__ ff, double* mq, double* cx, double* cy,
                            double* fa) {
  const int mm = m * m;
  const int64_t tot_v = E * mm, tot_f = E * 4 * m;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < tot_v + tot_f;
       g += (int64_t)gridDim.x * blockDim.x) {
    if (g < tot_v) {
      const int q = (int)(g % mm);
      const double w = wq[q % m] * wq[q / m];
      mq[g] = w * jdet[g];
      cx[g] = -dt * w * flux[g];
      cy[g] = -dt * w * flux[tot_v + g];
    } else {
      const int64_t gf = g - tot_v;
      fa[gf] = dt * wq[(int)(gf % m)] * ff[gf];
    }
  }
}

cudaError_t launch_metric_2d(const tpp_ctx* c, const double* jdet, const double* flux,
                             const double* ff, double dt, cudaStream_t s) {
  const double* wq = (c->mu > c->n) ? c->p<MuTables>(c->L.mutab)->w : c->p<Tables>(c->L.tables)->w;
  k_metric_2d<<<152 * 8, 256, 0, s>>>(wq, c->mu, c->E, dt, jdet, flux, ff, c->p<double>(c->L.mq),
                                      c->p<double>(c->L.cx), c->p<double>(c->L.cy),
                                      c->p<double>(c->L.fa));
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_precompute(const tpp_ctx* c, const double* vel_nodes,
                              const double* vel_face_normal, cudaStream_t s) {
  const bool d3 = c->dim == 3;
  const double* wq = (c->mu > c->n) ? c->p<MuTables>(c->L.mutab)->w : c->p<Tables>(c->L.tables)->w;
  k_precompute<<<152 * 8, 256, 0, s>>>(
      wq, c->dim, c->mu, c->E, c->prob.h, c->prob.dt, vel_nodes,
      vel_face_normal, c->p<double>(c->L.cx), c->p<double>(c->L.cy),
      d3 ? c->p<double>(c->L.cz) : nullptr, c->p<double>(c->L.fa));
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Face traces u(face node) = sum_i l_{0/1}[i] u_i along each direction.
// tr[e][f][t]: f = 0 (-x, l0), 1 (+x, l1), 2 (-y), 3 (+y) [, 4 (-z), 5 (+z)];
// t the face node (first tangential fastest).
template <int DIM, typename VT>
__global__ void k_traces(const Tables* T, int n, int64_t E, const VT* __restrict__ x,
                         VT* __restrict__ tr, const int32_t* skip) {
  if (skip && *skip) return;
  const int nfl = (DIM == 2) ? n : n * n;
  const int nloc = nfl * n;
  const int64_t tot = E * nfl;
  __shared__ VT l0[TPP_MAX_N], l1[TPP_MAX_N];
  if (threadIdx.x < n) {
    l0[threadIdx.x] = Tab<VT>::l0(T)[threadIdx.x];
    l1[threadIdx.x] = Tab<VT>::l1(T)[threadIdx.x];
  }
  __syncthreads();
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < tot;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / nfl;
    const int q = (int)(g % nfl);
    const int t0 = q % n, t1 = q / n;
    const VT* xe = x + e * nloc;
    VT* te = tr + e * (2 * DIM) * nfl;
    VT a0 = 0, a1 = 0, b0 = 0, b1 = 0, c0 = 0, c1 = 0;
    for (int s = 0; s < n; ++s) {
      // x-faces: tangential (y = t0, z = t1), sum over i = s
      const VT vx = (DIM == 2) ? xe[s + n * t0] : xe[s + n * t0 + n * n * t1];
      a0 += l0[s] * vx; a1 += l1[s] * vx;
      // y-faces: tangential (x = t0, z = t1), sum over j = s
      const VT vy = (DIM == 2) ? xe[t0 + n * s] : xe[t0 + n * s + n * n * t1];
      b0 += l0[s] * vy; b1 += l1[s] * vy;
      if (DIM == 3) {   // z-faces: tangential (x = t0, y = t1), sum over k = s
        const VT vz = xe[t0 + n * t1 + n * n * s];
        c0 += l0[s] * vz; c1 += l1[s] * vz;
      }
    }
    te[0 * nfl + q] = a0; te[1 * nfl + q] = a1;
    te[2 * nfl + q] = b0; te[3 * nfl + q] = b1;
    if (DIM == 3) { te[4 * nfl + q] = c0; te[5 * nfl + q] = c1; }
  }
}

cudaError_t launch_traces(const tpp_ctx* c, const double* x, double* tr, cudaStream_t s,
                          const int32_t* skip) {
  if (c->mu > c->n) return launch_traces_mu(c, x, tr, s, skip);
  if (c->dim == 2)
    k_traces<2, double><<<152 * 8, 256, 0, s>>>(c->p<Tables>(c->L.tables), c->n, c->EB, x, tr, skip);
  else
    k_traces<3, double><<<152 * 8, 256, 0, s>>>(c->p<Tables>(c->L.tables), c->n, c->EB, x, tr, skip);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_traces_f32(const tpp_ctx* c, const float* x, float* tr, cudaStream_t s,
                              const int32_t* skip) {
  if (c->mu > c->n) return launch_traces_mu_f32(c, x, tr, s, skip);
  if (c->dim == 2)
    k_traces<2, float><<<152 * 8, 256, 0, s>>>(c->p<Tables>(c->L.tables), c->n, c->EB, x, tr, skip);
  else
    k_traces<3, float><<<152 * 8, 256, 0, s>>>(c->p<Tables>(c->L.tables), c->n, c->EB, x, tr, skip);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// y = (M + dt A) x for one vector block per CTA (2D), Alg. matrix-free-matvec step 3:
//   y_ij = h^2 w_i w_j x_ij + sum_k D_ki cx_kj x_kj + sum_l D_lj cy_il x_il
//          + l0_i F_-x,j + l1_i F_+x,j + l0_j F_-y,i + l1_j F_+y,i,
// F_f = max(fa_f, 0) u^own_f + min(fa_f, 0) u^nbr_f the upwind flux out through face f
// (fa pre-scaled by dt h w); u^nbr_f is the trace of the neighbour's opposite face for
// the same right-hand side, and the inflow term is dropped where there is no
// neighbour.  Block b holds right-hand side b % R of element b / R.
template <typename VT>
__global__ void k_dg_apply_2d(const Tables* T, int n, VT hd, const VT* __restrict__ cx,
                              const VT* __restrict__ cy, const VT* __restrict__ fa,
                              const int32_t* __restrict__ nbr, const VT* __restrict__ x,
                              const VT* __restrict__ tr, VT* __restrict__ y, const int32_t* skip,
                              int R, const VT* __restrict__ mq) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smo[];
  VT* sm = reinterpret_cast<VT*>(smo);
  const int nn = n * n;
  VT* Ds = sm;                  // n*n, D[a*n + j]
  VT* px = Ds + nn;             // cx * x
  VT* py = px + nn;             // cy * x
  VT* fl = py + nn;             // 4n outward face fluxes, faces -x, +x, -y, +y
  VT* wl = fl + 4 * n;          // w, l0, l1
  const int64_t blk = blockIdx.x;                 // vector block
  const int64_t e = blk / R;                      // element (coefficients)
  const int r = (int)(blk % R);
  const int tid = threadIdx.x;
  const int64_t base = blk * nn, cbase = e * nn;
  for (int q = tid; q < nn; q += blockDim.x) {
    Ds[q] = Tab<VT>::D(T)[q];
    const VT xv = x[base + q];
    px[q] = cx[cbase + q] * xv;
    py[q] = cy[cbase + q] * xv;
  }
  if (tid < 4 * n) {
    const int f = tid / n, t = tid % n;
    const VT zero = (VT)0;
    const VT a = fa[(e * 4 + f) * n + t];
    const int64_t nb = nbr[e * 4 + f];
    VT F = max(a, zero) * tr[blk * 4 * n + f * n + t];
    if (nb >= 0) F += min(a, zero) * tr[((nb * R + r) * 4 + (f ^ 1)) * n + t];
    fl[f * n + t] = F;
  }
  if (tid < n) {
    wl[tid] = Tab<VT>::w(T)[tid];
    wl[n + tid] = Tab<VT>::l0(T)[tid];
    wl[2 * n + tid] = Tab<VT>::l1(T)[tid];
  }
  __syncthreads();
  const VT h2 = hd;                 // h^2
  for (int q = tid; q < nn; q += blockDim.x) {
    const int i = q % n, j = q / n;
    // mass: h^2 w_i w_j, or w |J_T| of a curved element (mq; hd = 0 drops it)
    const VT m = mq ? ((h2 != (VT)0) ? mq[cbase + q] : (VT)0) : h2 * wl[i] * wl[j];
    VT acc = m * x[base + q];
    for (int k = 0; k < n; ++k) acc += Ds[k * n + i] * px[k + n * j];
    for (int l = 0; l < n; ++l) acc += Ds[l * n + j] * py[i + n * l];
    acc += wl[n + i] * fl[j] + wl[2 * n + i] * fl[n + j];
    acc += wl[n + j] * fl[2 * n + i] + wl[2 * n + j] * fl[3 * n + i];
    y[base + q] = acc;
  }
}

// y = (M + dt A) x for one vector block per CTA (3D):
//   y_ijk = h^3 w_i w_j w_k x + sum_a D_ai cx_ajk x_ajk + sum_b D_bj cy_ibk x_ibk
//           + sum_c D_ck cz_ijc x_ijc + l0_i F_-x,jk + l1_i F_+x,jk + (same for y, z),
// outward face fluxes as in 2D, pre-scaled by dt h^2 and the two tangential weights.
template <typename VT>
__global__ void k_dg_apply_3d(const Tables* T, int n, VT hd, const VT* __restrict__ cx,
                              const VT* __restrict__ cy, const VT* __restrict__ cz,
                              const VT* __restrict__ fa, const int32_t* __restrict__ nbr,
                              const VT* __restrict__ x, const VT* __restrict__ tr,
                              VT* __restrict__ y, const int32_t* skip, int R) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smo[];
  VT* sm = reinterpret_cast<VT*>(smo);
  const int nn = n * n, n3 = nn * n;
  VT* Ds = sm;                  // n*n
  VT* px = Ds + nn;             // n^3 each
  VT* py = px + n3;
  VT* pz = py + n3;
  VT* fl = pz + n3;             // 6 n^2 outward fluxes: -x, +x, -y, +y, -z, +z
  VT* wl = fl + 6 * nn;         // w, l0, l1
  const int64_t blk = blockIdx.x;                 // vector block
  const int64_t e = blk / R;                      // element (coefficients)
  const int r = (int)(blk % R);
  const int tid = threadIdx.x;
  const int64_t base = blk * n3, cbase = e * n3;
  for (int q = tid; q < nn; q += blockDim.x) Ds[q] = Tab<VT>::D(T)[q];
  for (int q = tid; q < n3; q += blockDim.x) {
    const VT xv = x[base + q];
    px[q] = cx[cbase + q] * xv;
    py[q] = cy[cbase + q] * xv;
    pz[q] = cz[cbase + q] * xv;
  }
  if (tid < n) {
    wl[tid] = Tab<VT>::w(T)[tid];
    wl[n + tid] = Tab<VT>::l0(T)[tid];
    wl[2 * n + tid] = Tab<VT>::l1(T)[tid];
  }
  const VT zero = (VT)0;
  for (int g = tid; g < 6 * nn; g += blockDim.x) {
    const int f = g / nn, q = g % nn;
    const VT a = fa[(e * 6 + f) * nn + q];
    const int64_t nb = nbr[e * 6 + f];
    VT F = max(a, zero) * tr[blk * 6 * nn + f * nn + q];
    if (nb >= 0) F += min(a, zero) * tr[((nb * R + r) * 6 + (f ^ 1)) * nn + q];
    fl[g] = F;
  }
  __syncthreads();
  const VT h3 = hd;                 // h^3
  for (int q = tid; q < n3; q += blockDim.x) {
    const int i = q % n, j = (q / n) % n, k = q / nn;
    VT acc = h3 * wl[i] * wl[j] * wl[k] * x[base + q];
    for (int a = 0; a < n; ++a) acc += Ds[a * n + i] * px[a + n * j + nn * k];
    for (int b = 0; b < n; ++b) acc += Ds[b * n + j] * py[i + n * b + nn * k];
    for (int c = 0; c < n; ++c) acc += Ds[c * n + k] * pz[i + n * j + nn * c];
    const int qx = j + n * k, qy = i + n * k, qz = i + n * j;
    acc += wl[n + i] * fl[0 * nn + qx] + wl[2 * n + i] * fl[1 * nn + qx];
    acc += wl[n + j] * fl[2 * nn + qy] + wl[2 * n + j] * fl[3 * nn + qy];
    acc += wl[n + k] * fl[4 * nn + qz] + wl[2 * n + k] * fl[5 * nn + qz];
    y[base + q] = acc;
  }
}

template <typename VT>
cudaError_t launch_dg_apply_t(const tpp_ctx* c, const VT* cx, const VT* cy, const VT* cz,
                              const VT* fa, const VT* x, const VT* tr, VT* y,
                              const int32_t* skip, cudaStream_t s, double mass = 1.0,
                              const VT* mq = nullptr) {
  const int n = c->n;
  const int32_t* nbr = c->p<int32_t>(c->L.nbr);
  const double h = c->prob.h;
  if (c->dim == 2) {
    const int nn = n * n;
    int threads = ((nn + 31) / 32) * 32;
    if (threads < 4 * n) threads = ((4 * n + 31) / 32) * 32;
    const size_t smem = (3 * nn + 7 * n) * sizeof(VT);
    k_dg_apply_2d<VT><<<(unsigned)c->EB, threads, smem, s>>>(
        c->p<Tables>(c->L.tables), n, (VT)(mass * h * h), cx, cy, fa, nbr, x, tr, y, skip, c->R,
        mq);
    count_launch();
    return cudaGetLastError();
  }
  const int nn = n * n, n3 = nn * n;
  const size_t smem = (size_t)(nn + 3 * n3 + 6 * nn + 3 * n) * sizeof(VT);
  cudaError_t err = cudaFuncSetAttribute(k_dg_apply_3d<VT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_dg_apply_3d<VT><<<(unsigned)c->EB, 256, smem, s>>>(
      c->p<Tables>(c->L.tables), n, (VT)(mass * h * h * h), cx, cy, cz, fa, nbr, x, tr, y, skip,
      c->R);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_dg_apply(const tpp_ctx* c, const double* x, const double* tr, double* y,
                            const int32_t* skip, cudaStream_t s) {
  if (c->sys_nc > 0) return launch_sys_apply(c, x, tr, y, skip, s, 1.0);
  if (c->mu > c->n) return launch_dg_apply_mu(c, x, tr, y, skip, s, 1.0);
  const bool d3 = c->dim == 3;
  return launch_dg_apply_t<double>(c, c->p<double>(c->L.cx), c->p<double>(c->L.cy),
                                   d3 ? c->p<double>(c->L.cz) : nullptr, c->p<double>(c->L.fa),
                                   x, tr, y, skip, s, 1.0,
                                   c->curved ? c->p<double>(c->L.mq) : nullptr);
}

// y = dt A x = -dt J x: the operator without its mass term (traces tr of x given)
cudaError_t launch_dg_apply_flux(const tpp_ctx* c, const double* x, const double* tr, double* y,
                                 cudaStream_t s) {
  if (c->sys_nc > 0) return launch_sys_apply(c, x, tr, y, nullptr, s, 0.0);
  if (c->mu > c->n) return launch_dg_apply_mu(c, x, tr, y, nullptr, s, 0.0);
  const bool d3 = c->dim == 3;
  return launch_dg_apply_t<double>(c, c->p<double>(c->L.cx), c->p<double>(c->L.cy),
                                   d3 ? c->p<double>(c->L.cz) : nullptr, c->p<double>(c->L.fa),
                                   x, tr, y, nullptr, s, 0.0,
                                   c->curved ? c->p<double>(c->L.mq) : nullptr);
}

// FP32 operator (the inner solves of the mixed-precision mode) on the float
// copies of the flux Jacobian coefficients
cudaError_t launch_dg_apply_f32(const tpp_ctx* c, const float* x, const float* tr, float* y,
                                const int32_t* skip, cudaStream_t s) {
  if (c->mu > c->n) return launch_dg_apply_mu_f32(c, x, tr, y, skip, s);
  const float* f = c->p<float>(c->L.opf);
  const OpF32Layout O = op_f32_layout(c);
  return launch_dg_apply_t<float>(c, f + O.cx, f + O.cy, c->dim == 3 ? f + O.cz : nullptr,
                                  f + O.fa, x, tr, y, skip, s, 1.0,
                                  c->curved ? f + O.mq : nullptr);
}

// float copies of the operator coefficients (after k_precompute)
__global__ void k_op_to_f32(const double* cx, const double* cy, const double* cz,
                            const double* fa, const double* mq, float* out, OpF32Layout O,
                            int dim) {
  const int64_t tv = O.cy - O.cx, tf = O.tr - O.fa;
  const int64_t total = (int64_t)dim * tv + tf + (mq ? tv : 0);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    double v;
    size_t dst;
    if (g < dim * tv) {
      const int which = (int)(g / tv);
      const int64_t i = g % tv;
      v = (which == 0 ? cx : which == 1 ? cy : cz)[i];
      dst = (which == 0 ? O.cx : which == 1 ? O.cy : O.cz) + i;
    } else if (g < dim * tv + tf) {
      const int64_t i = g - dim * tv;
      v = fa[i];
      dst = O.fa + i;
    } else {                              // curved elements: the per-point mass
      const int64_t i = g - dim * tv - tf;
      v = mq[i];
      dst = O.mq + i;
    }
    out[dst] = __double2float_rn(v);
  }
}

cudaError_t launch_op_to_f32(const tpp_ctx* c, cudaStream_t s) {
  const OpF32Layout O = op_f32_layout(c);
  const bool d3 = c->dim == 3;
  k_op_to_f32<<<152 * 4, 256, 0, s>>>(c->p<double>(c->L.cx), c->p<double>(c->L.cy),
                                      d3 ? c->p<double>(c->L.cz) : nullptr,
                                      c->p<double>(c->L.fa),
                                      c->curved ? c->p<double>(c->L.mq) : nullptr,
                                      c->p<float>(c->L.opf), O, c->dim);
  count_launch();
  return cudaGetLastError();
}

}  // namespace tpp
