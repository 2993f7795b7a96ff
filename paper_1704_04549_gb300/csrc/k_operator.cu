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
  if (i < n) {
    const int k = n - 1 - i;                  // ascending order on [0, 1]
    double x = cos(M_PI * (k + 0.75) / (n + 0.5));
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
    {   // weight from the converged node
      double p0 = 1.0, p1 = x;
      for (int m = 2; m <= n; ++m) {
        const double p2 = ((2.0 * m - 1.0) * x * p1 - (m - 1.0) * p0) / m;
        p0 = p1;
        p1 = p2;
      }
      const double pn = (n == 1) ? x : p1;
      const double pm = (n == 1) ? 1.0 : p0;
      dp = n * (x * pn - pm) / (x * x - 1.0);
    }
    T->x[i] = 0.5 * (x + 1.0);
    T->w[i] = 1.0 / ((1.0 - x * x) * dp * dp);   // 2/(...) mapped by 1/2
  }
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
// dF_c/du = a_c, and for the upwind flux dF^/du^- = max(a.n, 0).  Stored
// pre-multiplied by the quadrature weights and metric factors:
//   cX[e][i + n j (+ n^2 k)] = -dt h^(d-1) w_i w_j (w_k) a_X(node)   (X = x, y, z)
//   sX[e][face node] = dt h^(d-1) (tangential weights) a_X(lower X-face node)
// The lower X-face of element e is owned by e; its upper X-face is the lower
// face of the +X neighbour, so both sides of a face read the same value.
// The field is a function of the normalised point x / L, L_d = nel_d h the
// domain length, so it is periodic on the mesh for any h.
__device__ __forceinline__ double vel_comp(const VelParams* V, int c, const double* X, int dim) {
  double a = V->a0[c];
  const int M = V->n_modes;
  for (int m = 0; m < M; ++m) {
    const double* k = V->kvec + (c * M + m) * dim;
    double kx = X[0] * k[0] + X[1] * k[1];
    if (dim == 3) kx += X[2] * k[2];
    a += V->amp[c * M + m] * cos(2.0 * M_PI * kx + V->phase[c * M + m]);
  }
  return a;
}

// Mesh mode: element (ex, ey, ez) of the periodic mesh, coordinates normalised
// by the domain length.  Batch mode (centres != NULL): element e is the cube of
// width h centred at centres[e], coordinates absolute in the unit domain, and
// the upper faces get their own values (sxu, syu, szu: no neighbour owns them).
__global__ void k_precompute(const VelParams* V, const Tables* T, int dim, int n, int nx, int ny,
                             int nz, double h, double dt, double* cx, double* cy, double* cz,
                             double* sx, double* sy, double* sz, const double* centres,
                             double* sxu, double* syu, double* szu, double span) {
  const int64_t E = centres ? (int64_t)nx : (int64_t)nx * ny * nz;
  const int nloc = (dim == 2) ? n * n : n * n * n;
  const int nfl = (dim == 2) ? n : n * n;
  const int64_t tot_v = E * nloc, tot_f = E * nfl;
  const double hf = (dim == 2) ? h : h * h;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < tot_v + tot_f;
       g += (int64_t)gridDim.x * blockDim.x) {
    if (g < tot_v) {
      const int64_t e = g / nloc;
      const int q = (int)(g % nloc);
      const int i = q % n, j = (q / n) % n, k = q / (n * n);
      double X[3];
      if (centres) {
        const double* ce = centres + e * dim;
        X[0] = ce[0] + span * (T->x[i] - 0.5);
        X[1] = ce[1] + span * (T->x[j] - 0.5);
        X[2] = (dim == 3) ? ce[2] + span * (T->x[k] - 0.5) : 0.0;
      } else {
        const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
        X[0] = (ex + T->x[i]) / nx;
        X[1] = (ey + T->x[j]) / ny;
        X[2] = (ez + T->x[k]) / nz;
      }
      double wq = T->w[i] * T->w[j];
      if (dim == 3) wq *= T->w[k];
      const double f = -dt * hf * wq;
      cx[g] = f * vel_comp(V, 0, X, dim);
      cy[g] = f * vel_comp(V, 1, X, dim);
      if (dim == 3) cz[g] = f * vel_comp(V, 2, X, dim);
    } else {
      const int64_t gf = g - tot_v;
      const int64_t e = gf / nfl;
      const int q = (int)(gf % nfl);
      const int t0 = q % n, t1 = q / n;   // tangential indices (first tangential fastest)
      const double wt = (dim == 2) ? T->w[t0] : T->w[t0] * T->w[t1];
      const double f = dt * hf * wt;
      if (centres) {
        const double* ce = centres + e * dim;
        const double lo[3] = {ce[0] - 0.5 * span, ce[1] - 0.5 * span,
                              dim == 3 ? ce[2] - 0.5 * span : 0.0};
        const double tx = span * T->x[t0], ty = span * T->x[t1];
        for (int up = 0; up < 2; ++up) {
          double Xx[3] = {lo[0] + up * span, lo[1] + tx, lo[2] + ty};  // x-face: (y, z)
          double Xy[3] = {lo[0] + tx, lo[1] + up * span, lo[2] + ty};  // y-face: (x, z)
          (up ? sxu : sx)[gf] = f * vel_comp(V, 0, Xx, dim);
          (up ? syu : sy)[gf] = f * vel_comp(V, 1, Xy, dim);
          if (dim == 3) {
            double Xz[3] = {lo[0] + tx, lo[1] + ty, lo[2] + up * span};   // z-face: (x, y)
            (up ? szu : sz)[gf] = f * vel_comp(V, 2, Xz, dim);
          }
        }
        continue;
      }
      const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
      {   // lower x-face: tangential (y, z)
        double X[3] = {(double)ex / nx, (ey + T->x[t0]) / ny, (ez + T->x[t1]) / nz};
        sx[gf] = f * vel_comp(V, 0, X, dim);
      }
      {   // lower y-face: tangential (x, z)
        double X[3] = {(ex + T->x[t0]) / nx, (double)ey / ny, (ez + T->x[t1]) / nz};
        sy[gf] = f * vel_comp(V, 1, X, dim);
      }
      if (dim == 3) {   // lower z-face: tangential (x, y)
        double X[3] = {(ex + T->x[t0]) / nx, (ey + T->x[t1]) / ny, (double)ez / nz};
        sz[gf] = f * vel_comp(V, 2, X, dim);
      }
    }
  }
}

cudaError_t launch_precompute(const tpp_ctx* c, cudaStream_t s) {
  const int nz = (c->dim == 3 && !c->iso) ? c->prob.nel[2] : 1;
  const bool d3 = c->dim == 3;
  k_precompute<<<152 * 8, 256, 0, s>>>(
      c->p<VelParams>(c->L.vel), c->p<Tables>(c->L.tables), c->dim, c->n,
      c->iso ? (int)c->E : c->prob.nel[0], c->iso ? 1 : c->prob.nel[1], nz, c->prob.h,
      c->prob.dt, c->p<double>(c->L.cx), c->p<double>(c->L.cy),
      d3 ? c->p<double>(c->L.cz) : nullptr, c->p<double>(c->L.sx), c->p<double>(c->L.sy),
      d3 ? c->p<double>(c->L.sz) : nullptr, c->iso ? c->p<double>(c->L.centres) : nullptr,
      c->iso ? c->p<double>(c->L.sxu) : nullptr, c->iso ? c->p<double>(c->L.syu) : nullptr,
      (c->iso && d3) ? c->p<double>(c->L.szu) : nullptr,
      c->prob.batch_span > 0.0 ? c->prob.batch_span : c->prob.h);
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
  if (c->dim == 2)
    k_traces<2, double><<<152 * 8, 256, 0, s>>>(c->p<Tables>(c->L.tables), c->n, c->EB, x, tr, skip);
  else
    k_traces<3, double><<<152 * 8, 256, 0, s>>>(c->p<Tables>(c->L.tables), c->n, c->EB, x, tr, skip);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_traces_f32(const tpp_ctx* c, const float* x, float* tr, cudaStream_t s,
                              const int32_t* skip) {
  if (c->dim == 2)
    k_traces<2, float><<<152 * 8, 256, 0, s>>>(c->p<Tables>(c->L.tables), c->n, c->EB, x, tr, skip);
  else
    k_traces<3, float><<<152 * 8, 256, 0, s>>>(c->p<Tables>(c->L.tables), c->n, c->EB, x, tr, skip);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// y = (M + dt A) x for one element per CTA (2D), Alg. matrix-free-matvec step 3:
//   y_ij = h^2 w_i w_j x_ij + sum_k D_ki cx_kj x_kj + sum_l D_lj cy_il x_il
//          + l1_i F^R_j - l0_i F^L_j + l1_j F^T_i - l0_j F^B_i,
// F^R_j = max(sR_j,0) u^-_R + min(sR_j,0) u^+_R (upwind flux through the +x
// face, pre-scaled by dt h w_j), etc.
// Batch mode (R >= 1 right-hand sides per isolated element, sxu / syu given):
// block b holds rhs b % R of element b / R; only the own-side upwind face terms
// (outflow through each face) remain.
template <typename VT>
__global__ void k_dg_apply_2d(const Tables* T, int n, int nx, int ny, VT hd,
                              const VT* __restrict__ cx, const VT* __restrict__ cy,
                              const VT* __restrict__ sx, const VT* __restrict__ sy,
                              const VT* __restrict__ x, const VT* __restrict__ tr,
                              VT* __restrict__ y, const int32_t* skip, int R,
                              const VT* __restrict__ sxu, const VT* __restrict__ syu) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smo[];
  VT* sm = reinterpret_cast<VT*>(smo);
  const int nn = n * n;
  VT* Ds = sm;                  // n*n, D[a*n + j]
  VT* px = Ds + nn;             // cx * x
  VT* py = px + nn;             // cy * x
  VT* fl = py + nn;             // 4n face fluxes: R, L, T, B
  VT* wl = fl + 4 * n;          // w, l0, l1
  const int64_t blk = blockIdx.x;                 // vector block
  const bool iso = sxu != nullptr;
  const int64_t e = iso ? blk / R : blk;           // element (coefficients)
  const int ex = (int)(e % nx), ey = (int)(e / nx);
  const int64_t eR = ey * (int64_t)nx + (ex + 1) % nx, eL = ey * (int64_t)nx + (ex + nx - 1) % nx;
  const int64_t eT = ((ey + 1) % ny) * (int64_t)nx + ex, eB = ((ey + ny - 1) % ny) * (int64_t)nx + ex;
  const int tid = threadIdx.x;
  const int64_t base = blk * nn, cbase = e * nn;
  for (int q = tid; q < nn; q += blockDim.x) {
    Ds[q] = Tab<VT>::D(T)[q];
    const VT xv = x[base + q];
    px[q] = cx[cbase + q] * xv;
    py[q] = cy[cbase + q] * xv;
  }
  if (tid < n) {
    wl[tid] = Tab<VT>::w(T)[tid];
    wl[n + tid] = Tab<VT>::l0(T)[tid];
    wl[2 * n + tid] = Tab<VT>::l1(T)[tid];
    const VT* te = tr + blk * 4 * n;
    const int t = tid;
    const VT zero = (VT)0;
    if (iso) {   // own traces only: outflow through each face
      fl[t] = max(sxu[e * n + t], zero) * te[1 * n + t];
      fl[n + t] = min(sx[e * n + t], zero) * te[0 * n + t];
      fl[2 * n + t] = max(syu[e * n + t], zero) * te[3 * n + t];
      fl[3 * n + t] = min(sy[e * n + t], zero) * te[2 * n + t];
    } else {
    {   // +x face: outward normal +x, flux a_x evaluated on the face owned by eR
      const VT s = sx[eR * n + t];
      fl[t] = max(s, zero) * te[1 * n + t] + min(s, zero) * tr[eR * 4 * n + 0 * n + t];
    }
    {   // -x face: flux through it in the +x direction, from the left element
      const VT s = sx[e * n + t];
      fl[n + t] = max(s, zero) * tr[eL * 4 * n + 1 * n + t] + min(s, zero) * te[0 * n + t];
    }
    {   // +y
      const VT s = sy[eT * n + t];
      fl[2 * n + t] = max(s, zero) * te[3 * n + t] + min(s, zero) * tr[eT * 4 * n + 2 * n + t];
    }
    {   // -y
      const VT s = sy[e * n + t];
      fl[3 * n + t] = max(s, zero) * tr[eB * 4 * n + 3 * n + t] + min(s, zero) * te[2 * n + t];
    }
    }
  }
  __syncthreads();
  const VT h2 = hd;                 // h^2
  for (int q = tid; q < nn; q += blockDim.x) {
    const int i = q % n, j = q / n;
    VT acc = h2 * wl[i] * wl[j] * x[base + q];
    for (int k = 0; k < n; ++k) acc += Ds[k * n + i] * px[k + n * j];
    for (int l = 0; l < n; ++l) acc += Ds[l * n + j] * py[i + n * l];
    acc += wl[2 * n + i] * fl[j] - wl[n + i] * fl[n + j];
    acc += wl[2 * n + j] * fl[2 * n + i] - wl[n + j] * fl[3 * n + i];
    y[base + q] = acc;
  }
}

// y = (M + dt A) x for one element per CTA (3D):
//   y_ijk = h^3 w_i w_j w_k x + sum_a D_ai cx_ajk x_ajk + sum_b D_bj cy_ibk x_ibk
//           + sum_c D_ck cz_ijc x_ijc + l1_i F^+x_jk - l0_i F^-x_jk + (same for y, z),
// face fluxes pre-scaled by dt h^2 and the two tangential weights.
template <typename VT>
__global__ void k_dg_apply_3d(const Tables* T, int n, int nx, int ny, int nz, VT hd,
                              const VT* __restrict__ cx, const VT* __restrict__ cy,
                              const VT* __restrict__ cz, const VT* __restrict__ sx,
                              const VT* __restrict__ sy, const VT* __restrict__ sz,
                              const VT* __restrict__ x, const VT* __restrict__ tr,
                              VT* __restrict__ y, const int32_t* skip, int R,
                              const VT* __restrict__ sxu, const VT* __restrict__ syu,
                              const VT* __restrict__ szu) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smo[];
  VT* sm = reinterpret_cast<VT*>(smo);
  const int nn = n * n, n3 = nn * n;
  VT* Ds = sm;                  // n*n
  VT* px = Ds + nn;             // n^3 each
  VT* py = px + n3;
  VT* pz = py + n3;
  VT* fl = pz + n3;             // 6 n^2 fluxes: +x, -x, +y, -y, +z, -z
  VT* wl = fl + 6 * nn;         // w, l0, l1
  const int64_t blk = blockIdx.x;                 // vector block
  const bool iso = sxu != nullptr;
  const int64_t e = iso ? blk / R : blk;           // element (coefficients)
  const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
  auto eid = [&](int a, int b, int c) -> int64_t {
    return ((int64_t)((c + nz) % nz) * ny + (b + ny) % ny) * nx + (a + nx) % nx;
  };
  const int64_t eXp = eid(ex + 1, ey, ez), eXm = eid(ex - 1, ey, ez);
  const int64_t eYp = eid(ex, ey + 1, ez), eYm = eid(ex, ey - 1, ez);
  const int64_t eZp = eid(ex, ey, ez + 1), eZm = eid(ex, ey, ez - 1);
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
  const VT* te = tr + blk * 6 * nn;
  const VT zero = (VT)0;
  if (iso) {   // own traces only: outflow through each face
    for (int q = tid; q < nn; q += blockDim.x) {
      fl[0 * nn + q] = max(sxu[e * nn + q], zero) * te[1 * nn + q];
      fl[1 * nn + q] = min(sx[e * nn + q], zero) * te[0 * nn + q];
      fl[2 * nn + q] = max(syu[e * nn + q], zero) * te[3 * nn + q];
      fl[3 * nn + q] = min(sy[e * nn + q], zero) * te[2 * nn + q];
      fl[4 * nn + q] = max(szu[e * nn + q], zero) * te[5 * nn + q];
      fl[5 * nn + q] = min(sz[e * nn + q], zero) * te[4 * nn + q];
    }
  } else
  for (int q = tid; q < nn; q += blockDim.x) {
    VT s;
    s = sx[eXp * nn + q];
    fl[0 * nn + q] = max(s, zero) * te[1 * nn + q] + min(s, zero) * tr[eXp * 6 * nn + 0 * nn + q];
    s = sx[e * nn + q];
    fl[1 * nn + q] = max(s, zero) * tr[eXm * 6 * nn + 1 * nn + q] + min(s, zero) * te[0 * nn + q];
    s = sy[eYp * nn + q];
    fl[2 * nn + q] = max(s, zero) * te[3 * nn + q] + min(s, zero) * tr[eYp * 6 * nn + 2 * nn + q];
    s = sy[e * nn + q];
    fl[3 * nn + q] = max(s, zero) * tr[eYm * 6 * nn + 3 * nn + q] + min(s, zero) * te[2 * nn + q];
    s = sz[eZp * nn + q];
    fl[4 * nn + q] = max(s, zero) * te[5 * nn + q] + min(s, zero) * tr[eZp * 6 * nn + 4 * nn + q];
    s = sz[e * nn + q];
    fl[5 * nn + q] = max(s, zero) * tr[eZm * 6 * nn + 5 * nn + q] + min(s, zero) * te[4 * nn + q];
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
    acc += wl[2 * n + i] * fl[0 * nn + qx] - wl[n + i] * fl[1 * nn + qx];
    acc += wl[2 * n + j] * fl[2 * nn + qy] - wl[n + j] * fl[3 * nn + qy];
    acc += wl[2 * n + k] * fl[4 * nn + qz] - wl[n + k] * fl[5 * nn + qz];
    y[base + q] = acc;
  }
}

template <typename VT>
cudaError_t launch_dg_apply_t(const tpp_ctx* c, const VT* cx, const VT* cy, const VT* cz,
                              const VT* sx, const VT* sy, const VT* sz, const VT* sxu,
                              const VT* syu, const VT* szu, const VT* x, const VT* tr, VT* y,
                              const int32_t* skip, cudaStream_t s) {
  const int n = c->n;
  if (c->dim == 2) {
    const int nn = n * n;
    const int threads = ((nn + 31) / 32) * 32;
    const size_t smem = (3 * nn + 7 * n) * sizeof(VT);
    const double h = c->prob.h;
    k_dg_apply_2d<VT><<<(unsigned)c->EB, threads, smem, s>>>(
        c->p<Tables>(c->L.tables), n, c->iso ? (int)c->E : c->prob.nel[0],
        c->iso ? 1 : c->prob.nel[1], (VT)(h * h), cx, cy, sx, sy, x, tr, y, skip, c->R,
        c->iso ? sxu : nullptr, c->iso ? syu : nullptr);
    count_launch();
    return cudaGetLastError();
  }
  const int nn = n * n, n3 = nn * n;
  const size_t smem = (size_t)(nn + 3 * n3 + 6 * nn + 3 * n) * sizeof(VT);
  cudaError_t err = cudaFuncSetAttribute(k_dg_apply_3d<VT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const double h = c->prob.h;
  k_dg_apply_3d<VT><<<(unsigned)c->EB, 256, smem, s>>>(
      c->p<Tables>(c->L.tables), n, c->iso ? (int)c->E : c->prob.nel[0],
      c->iso ? 1 : c->prob.nel[1], c->iso ? 1 : c->prob.nel[2], (VT)(h * h * h), cx, cy, cz, sx,
      sy, sz, x, tr, y, skip, c->R, c->iso ? sxu : nullptr, c->iso ? syu : nullptr,
      c->iso ? szu : nullptr);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_dg_apply(const tpp_ctx* c, const double* x, const double* tr, double* y,
                            const int32_t* skip, cudaStream_t s) {
  const bool d3 = c->dim == 3;
  return launch_dg_apply_t<double>(
      c, c->p<double>(c->L.cx), c->p<double>(c->L.cy), d3 ? c->p<double>(c->L.cz) : nullptr,
      c->p<double>(c->L.sx), c->p<double>(c->L.sy), d3 ? c->p<double>(c->L.sz) : nullptr,
      c->iso ? c->p<double>(c->L.sxu) : nullptr, c->iso ? c->p<double>(c->L.syu) : nullptr,
      (c->iso && d3) ? c->p<double>(c->L.szu) : nullptr, x, tr, y, skip, s);
}

// FP32 operator (the inner solves of the mixed-precision mode) on the float
// copies of the flux Jacobian coefficients
cudaError_t launch_dg_apply_f32(const tpp_ctx* c, const float* x, const float* tr, float* y,
                                const int32_t* skip, cudaStream_t s) {
  const float* f = c->p<float>(c->L.opf);
  const OpF32Layout O = op_f32_layout(c);
  const bool d3 = c->dim == 3;
  return launch_dg_apply_t<float>(c, f + O.cx, f + O.cy, d3 ? f + O.cz : nullptr, f + O.sx,
                                  f + O.sy, d3 ? f + O.sz : nullptr, f + O.sxu, f + O.syu,
                                  f + O.szu, x, tr, y, skip, s);
}

// float copies of the operator coefficients (after k_precompute)
__global__ void k_op_to_f32(const double* cx, const double* cy, const double* cz,
                            const double* sx, const double* sy, const double* sz,
                            const double* sxu, const double* syu, const double* szu, float* out,
                            OpF32Layout O, int dim, int iso) {
  const int64_t tv = O.cy - O.cx, tf = O.sy - O.sx;
  const int nface = iso ? 2 * dim : dim;
  const int64_t total = (int64_t)dim * tv + nface * tf;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    double v;
    size_t dst;
    if (g < dim * tv) {
      const int which = (int)(g / tv);
      const int64_t i = g % tv;
      v = (which == 0 ? cx : which == 1 ? cy : cz)[i];
      dst = (which == 0 ? O.cx : which == 1 ? O.cy : O.cz) + i;
    } else {
      const int64_t h = g - dim * tv;
      const int which = (int)(h / tf);           // sx, sy, (sz,) then sxu, syu, (szu)
      const int64_t i = h % tf;
      const int dir = which % dim, up = which / dim;
      const double* src = up ? (dir == 0 ? sxu : dir == 1 ? syu : szu)
                             : (dir == 0 ? sx : dir == 1 ? sy : sz);
      v = src[i];
      dst = (up ? (dir == 0 ? O.sxu : dir == 1 ? O.syu : O.szu)
                : (dir == 0 ? O.sx : dir == 1 ? O.sy : O.sz)) + i;
    }
    out[dst] = __double2float_rn(v);
  }
}

cudaError_t launch_op_to_f32(const tpp_ctx* c, cudaStream_t s) {
  const OpF32Layout O = op_f32_layout(c);
  const bool d3 = c->dim == 3;
  k_op_to_f32<<<152 * 4, 256, 0, s>>>(
      c->p<double>(c->L.cx), c->p<double>(c->L.cy), d3 ? c->p<double>(c->L.cz) : nullptr,
      c->p<double>(c->L.sx), c->p<double>(c->L.sy), d3 ? c->p<double>(c->L.sz) : nullptr,
      c->iso ? c->p<double>(c->L.sxu) : nullptr, c->iso ? c->p<double>(c->L.syu) : nullptr,
      (c->iso && d3) ? c->p<double>(c->L.szu) : nullptr, c->p<float>(c->L.opf), O, c->dim,
      c->iso ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

}  // namespace tpp
