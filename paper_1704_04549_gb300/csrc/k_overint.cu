// Over-integration (mu > n quadrature points per direction, 2D): Sec. 3.2's G and D
// at the mu-point Gauss-Legendre rule, the sum-factorised operator through those
// points (Table tab:dg-ops, Alg. matrix-free-matvec step 3) and the explicit KSVD
// core of the rearranged block (Sec. 4.1 / 4.2.1).
//
// Structure of the rearranged block.  Every term of the element block is a sum over
// quadrature points of Kronecker products of rank-one 1D matrices: with g_b, d_b the
// rows of G and D at point b and l0, l1 the endpoint values,
//   mass         sum_ab h^2 w_a w_b (g_b g_b^T) (x) (g_a g_a^T)
//   x-volume     sum_ab cx(a,b) (g_b g_b^T) (x) (d_a g_a^T)
//   y-volume     sum_ab cy(a,b) (d_b g_b^T) (x) (g_a g_a^T)
//   x-faces      sum_b max(fa_{+-x}(b), 0) (g_b g_b^T) (x) (l l^T)
//   y-faces      sum_a max(fa_{+-y}(a), 0) (l l^T) (x) (g_a g_a^T)
// (left factor y, right factor x), so its Van Loan-Pitsianis rearrangement is
// A~ = B K B^T with the element-independent basis
//   B = [vec(g_b g_b^T) (b < mu) | vec(d_b g_b^T) (b < mu) | vec(l1 l1^T) | vec(l0 l0^T)]
// (n^2 x (2 mu + 2)) and a per-element K of the weights and flux Jacobians at the
// quadrature points.  One Householder QR B = Q R per context gives
// A~ = Q (R K R^T) Q^T: the top singular triplets of A~ are those of the small core
// R K R^T, mapped by Q (exact, O(mu^3) per element).
#include <string>

#include "tpp_internal.cuh"

namespace tpp {

namespace {

// the mu-point rule and the nodal basis (n nodes) at its points: G by the product
// formula, D by phi_j' = phi_j sum_{m != j} 1 / (xi - x_m) away from the nodes and the
// nodal differentiation matrix at a node
__global__ void k_mu_tables(const Tables* T, int n, int mu, MuTables* M) {
  __shared__ double lam[TPP_MAX_N];
  const int t = threadIdx.x;
  if (t < mu) gauss_legendre_node(mu, t, &M->x[t], &M->w[t]);
  if (t < n) {
    double prod = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != t) prod *= (T->x[t] - T->x[m]);
    lam[t] = 1.0 / prod;
  }
  __syncthreads();
  if (t < mu) {
    const double xi = M->x[t];
    int hit = -1;
    for (int m = 0; m < n; ++m)
      if (xi == T->x[m]) hit = m;
    for (int j = 0; j < n; ++j) {
      double g, d;
      if (hit >= 0) {
        g = (j == hit) ? 1.0 : 0.0;
        d = T->D[hit * n + j];
      } else {
        double prod = lam[j], sinv = 0.0;
        for (int m = 0; m < n; ++m)
          if (m != j) {
            prod *= (xi - T->x[m]);
            sinv += 1.0 / (xi - T->x[m]);
          }
        g = prod;
        d = prod * sinv;
      }
      M->G[t * n + j] = g;
      M->D[t * n + j] = d;
      M->Gf[t * n + j] = __double2float_rn(g);
      M->Df[t * n + j] = __double2float_rn(d);
    }
  }
  if (t < n) M->wf[t] = __double2float_rn(T->w[t]);
}

// B (column-major n^2 x m, m = 2 mu + 2) and its Householder QR: Q (n^2 x p, p =
// min(n^2, m)), R (p x m, row-major), qtr[t] = trace of mat(Q[:, t]).  One CTA.
__global__ void k_mu_basis(const Tables* T, const MuTables* M, int n, int mu, double* W,
                           double* tau, double* Q, double* Rb, double* qtr) {
  __shared__ double red[32];
  const int nn = n * n, m = 2 * mu + 2, p = (nn < m) ? nn : m;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int q = tid; q < nn * m; q += nt) {
    const int row = q % nn, col = q / nn;
    const int j = row % n, l = row / n;
    double v;
    if (col < mu) v = M->G[col * n + j] * M->G[col * n + l];
    else if (col < 2 * mu) v = M->D[(col - mu) * n + j] * M->G[(col - mu) * n + l];
    else if (col == 2 * mu) v = T->l1[j] * T->l1[l];
    else v = T->l0[j] * T->l0[l];
    W[q] = v;
  }
  __syncthreads();
  for (int k = 0; k < p; ++k) {
    double* col = W + (size_t)k * nn;
    double s2 = 0.0;
    for (int i = k + 1 + tid; i < nn; i += nt) s2 += col[i] * col[i];
    s2 = block_sum(s2, red);
    const double x0 = col[k];
    double t = 0.0, alpha = x0;
    if (s2 > 0.0) {
      const double nx = sqrt(x0 * x0 + s2);
      alpha = (x0 > 0.0) ? -nx : nx;
      t = (alpha - x0) / alpha;
    }
    __syncthreads();
    if (s2 > 0.0) {
      const double iv = 1.0 / (x0 - alpha);
      for (int i = k + 1 + tid; i < nn; i += nt) col[i] *= iv;   // v = (1, col[k+1:])
    }
    __syncthreads();
    if (tid == 0) {
      col[k] = alpha;
      tau[k] = t;
    }
    for (int c = k + 1 + wid; c < m; c += nw) {      // H_k applied to the later columns
      double* cj = W + (size_t)c * nn;
      double sv = 0.0;
      for (int i = k + 1 + lane; i < nn; i += 32) sv += col[i] * cj[i];
      sv = warp_sum(sv);
      sv = t * (sv + cj[k]);
      __syncwarp();
      if (lane == 0) cj[k] -= sv;
      for (int i = k + 1 + lane; i < nn; i += 32) cj[i] -= sv * col[i];
    }
    __syncthreads();
  }
  for (int q = tid; q < p * m; q += nt) {
    const int r = q / m, c = q % m;
    Rb[q] = (c >= r) ? W[(size_t)c * nn + r] : 0.0;
  }
  for (int q = tid; q < nn * p; q += nt) {
    const int row = q % nn, c = q / nn;
    Q[q] = (row == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = p - 1; k >= 0; --k) {                   // Q = H_0 ... H_{p-1} I[:, :p]
    const double* v = W + (size_t)k * nn;
    const double t = tau[k];
    for (int c = k + wid; c < p; c += nw) {
      double* qc = Q + (size_t)c * nn;
      double sv = 0.0;
      for (int i = k + 1 + lane; i < nn; i += 32) sv += v[i] * qc[i];
      sv = warp_sum(sv) + qc[k];
      __syncwarp();
      const double f = t * sv;
      if (lane == 0) qc[k] -= f;
      for (int i = k + 1 + lane; i < nn; i += 32) qc[i] -= f * v[i];
    }
    __syncthreads();
  }
  for (int c = tid; c < p; c += nt) {
    double sv = 0.0;
    for (int a = 0; a < n; ++a) sv += Q[(size_t)c * nn + a * (n + 1)];
    qtr[c] = sv;
  }
}

// core R K R^T (column-major p x p) of every element; one CTA per element, K and
// K R^T in shared memory
__global__ void __launch_bounds__(128)
k_core_mu(int n, int mu, int64_t E, double h, const MuTables* M, const double* __restrict__ cx,
          const double* __restrict__ cy, const double* __restrict__ fa,
          const double* __restrict__ Rb, double* __restrict__ cores,
          const double* __restrict__ mq) {
  extern __shared__ double smc[];
  const int nn = n * n, m = 2 * mu + 2, p = (nn < m) ? nn : m;
  const int64_t e = blockIdx.x;
  double* K = smc;                 // m x m, row-major
  double* KR = K + m * m;          // m x p: K R^T
  const int tid = threadIdx.x, nt = blockDim.x;
  const double* cxe = cx + e * mu * mu;
  const double* cye = cy + e * mu * mu;
  const double* fe = fa + e * 4 * mu;     // faces -x, +x, -y, +y
  for (int q = tid; q < m * m; q += nt) {
    const int row = q / m, col = q % m;
    double v = 0.0;
    if (row < mu) {
      const int b = row;
      if (col < mu)                                                  // mass (curved: w |J_T|)
        v = mq ? mq[e * mu * mu + col + mu * b] : h * h * M->w[col] * M->w[b];
      else if (col < 2 * mu) v = cxe[(col - mu) + mu * b];           // x-volume
      else if (col == 2 * mu) v = fmax(fe[1 * mu + b], 0.0);         // +x face
      else v = fmax(fe[0 * mu + b], 0.0);                            // -x face
    } else if (row < 2 * mu) {
      if (col < mu) v = cye[col + mu * (row - mu)];                  // y-volume
    } else if (col < mu) {
      v = fmax(fe[(row == 2 * mu ? 3 : 2) * mu + col], 0.0);         // +y / -y faces
    }
    K[q] = v;
  }
  __syncthreads();
  for (int q = tid; q < m * p; q += nt) {          // KR[row][c] = sum_k K[row][k] R[c][k]
    const int row = q / p, c = q % p;
    double sv = 0.0;
    for (int k = c; k < m; ++k) sv += K[row * m + k] * Rb[c * m + k];   // R upper trapezoidal
    KR[q] = sv;
  }
  __syncthreads();
  double* out = cores + e * p * p;
  for (int q = tid; q < p * p; q += nt) {          // core[r][c] = sum_k R[r][k] KR[k][c]
    const int r = q % p, c = q / p;
    double sv = 0.0;
    for (int k = r; k < m; ++k) sv += Rb[r * m + k] * KR[k * p + c];
    out[q] = sv;                                    // column-major (r + p c)
  }
}

// face traces at the mu tangential points: tr[blk][f][t], f = -x, +x, -y, +y
template <typename VT>
__global__ void k_traces_mu(const Tables* T, const MuTables* M, int n, int mu, int64_t EB,
                            const VT* __restrict__ x, VT* __restrict__ tr, const int32_t* skip) {
  if (skip && *skip) return;
  const int nn = n * n;
  const int64_t tot = EB * 4 * mu;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < tot;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = g / (4 * mu);
    const int f = (int)((g / mu) % 4), t = (int)(g % mu);
    const VT* xe = x + blk * nn;
    const double* l = (f & 1) ? T->l1 : T->l0;
    double sv = 0.0;
    if (f < 2) {                       // x-face: tangential y
      for (int j = 0; j < n; ++j) {
        double ej = 0.0;
        for (int i = 0; i < n; ++i) ej += l[i] * (double)xe[i + n * j];
        sv += M->G[t * n + j] * ej;
      }
    } else {                           // y-face: tangential x
      for (int i = 0; i < n; ++i) {
        double ei = 0.0;
        for (int j = 0; j < n; ++j) ei += l[j] * (double)xe[i + n * j];
        sv += M->G[t * n + i] * ei;
      }
    }
    tr[g] = (VT)sv;
  }
}

// y = (mass) M x + dt A x through the mu-point rule, one vector block per CTA
template <typename VT>
__global__ void __launch_bounds__(256)
k_dg_apply_mu(const Tables* T, const MuTables* M, int n, int mu, double mass_h2,
              const VT* __restrict__ cx, const VT* __restrict__ cy, const VT* __restrict__ fa,
              const int32_t* __restrict__ nbr, const VT* __restrict__ x,
              const VT* __restrict__ tr, VT* __restrict__ y, const int32_t* skip, int R,
              const VT* __restrict__ mq) {
  if (skip && *skip) return;
  // curved elements: the mass goes through the mu-point rule, w |J_T| u at the points
  const bool qmass = mq && mass_h2 != 0.0;
  extern __shared__ __align__(16) unsigned char smo[];
  VT* sm = reinterpret_cast<VT*>(smo);
  const int nn = n * n, qq = mu * mu;
  VT* G = sm;                 // mu n
  VT* D = G + mu * n;         // mu n
  VT* xs = D + mu * n;        // n^2
  VT* t1 = xs + nn;           // n mu
  VT* t2 = t1 + n * mu;       // n mu
  VT* px = t2 + n * mu;       // mu^2
  VT* py = px + qq;           // mu^2
  VT* fl = py + qq;           // 4 mu outward fluxes
  VT* pm = fl + 4 * mu;       // mu^2 (curved mass)
  const int64_t blk = blockIdx.x, e = blk / R;
  const int r = (int)(blk % R);
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int q = tid; q < mu * n; q += nt) {
    G[q] = (VT)M->G[q];
    D[q] = (VT)M->D[q];
  }
  for (int q = tid; q < nn; q += nt) xs[q] = x[blk * nn + q];
  for (int q = tid; q < 4 * mu; q += nt) {
    const int f = q / mu, t = q % mu;
    const VT a = fa[(e * 4 + f) * mu + t];
    const int64_t nb = nbr[e * 4 + f];
    const VT zero = (VT)0;
    VT F = max(a, zero) * tr[(blk * 4 + f) * mu + t];
    if (nb >= 0) F += min(a, zero) * tr[((nb * R + r) * 4 + (f ^ 1)) * mu + t];
    fl[q] = F;
  }
  __syncthreads();
  // u at the quadrature points: t1[i + n b] = sum_j G[b][j] x[i + n j], u = G t1
  for (int q = tid; q < n * mu; q += nt) {
    const int i = q % n, b = q / n;
    VT s = 0;
    for (int j = 0; j < n; ++j) s += G[b * n + j] * xs[i + n * j];
    t1[q] = s;
  }
  __syncthreads();
  for (int q = tid; q < qq; q += nt) {
    const int a = q % mu, b = q / mu;
    VT s = 0;
    for (int i = 0; i < n; ++i) s += G[a * n + i] * t1[i + n * b];
    px[q] = cx[e * qq + q] * s;
    py[q] = cy[e * qq + q] * s;
    if (qmass) pm[q] = mq[e * qq + q] * s;
  }
  __syncthreads();
  // t1[i + n b] = sum_a D[a][i] px[a + mu b];  t2[i + n b] = sum_a G[a][i] py[a + mu b]
  for (int q = tid; q < n * mu; q += nt) {
    const int i = q % n, b = q / n;
    VT s1 = 0, s2 = 0;
    for (int a = 0; a < mu; ++a) {
      s1 += D[a * n + i] * px[a + mu * b];
      s2 += G[a * n + i] * py[a + mu * b];
    }
    if (qmass)
      for (int a = 0; a < mu; ++a) s1 += G[a * n + i] * pm[a + mu * b];
    t1[q] = s1;
    t2[q] = s2;
  }
  __syncthreads();
  for (int q = tid; q < nn; q += nt) {
    const int i = q % n, j = q / n;
    VT acc = qmass ? (VT)0 : (VT)(mass_h2 * T->w[i] * T->w[j]) * xs[q];
    VT fx0 = 0, fx1 = 0, fy0 = 0, fy1 = 0;
    for (int b = 0; b < mu; ++b) {
      acc += G[b * n + j] * t1[i + n * b] + D[b * n + j] * t2[i + n * b];
      fx0 += G[b * n + j] * fl[0 * mu + b];
      fx1 += G[b * n + j] * fl[1 * mu + b];
      fy0 += G[b * n + i] * fl[2 * mu + b];
      fy1 += G[b * n + i] * fl[3 * mu + b];
    }
    acc += (VT)T->l0[i] * fx0 + (VT)T->l1[i] * fx1 + (VT)T->l0[j] * fy0 + (VT)T->l1[j] * fy1;
    y[blk * nn + q] = acc;
  }
}

template <typename VT>
cudaError_t dg_apply_mu_t(const tpp_ctx* c, const VT* cx, const VT* cy, const VT* fa,
                          const VT* x, const VT* tr, VT* y, const int32_t* skip, cudaStream_t s,
                          double mass, const VT* mq) {
  const int n = c->n, mu = c->mu;
  const size_t smem =
      (size_t)(2 * mu * n + n * n + 2 * n * mu + 3 * mu * mu + 4 * mu) * sizeof(VT);
  cudaError_t e = cudaFuncSetAttribute(k_dg_apply_mu<VT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_dg_apply_mu<VT><<<(unsigned)c->EB, 256, smem, s>>>(
      c->p<Tables>(c->L.tables), c->p<MuTables>(c->L.mutab), n, mu,
      mass * c->prob.h * c->prob.h, cx, cy, fa, c->p<int32_t>(c->L.nbr), x, tr, y, skip, c->R,
      mq);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mu_setup(const tpp_ctx* c, cudaStream_t s) {
  MuTables* M = c->p<MuTables>(c->L.mutab);
  k_mu_tables<<<1, 64, 0, s>>>(c->p<Tables>(c->L.tables), c->n, c->mu, M);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nn = c->n * c->n, m = 2 * c->mu + 2;
  double* W = c->p<double>(c->L.bwork);
  k_mu_basis<<<1, 1024, 0, s>>>(c->p<Tables>(c->L.tables), M, c->n, c->mu, W,
                                W + (size_t)nn * m, c->p<double>(c->L.qb), c->p<double>(c->L.rb),
                                c->p<double>(c->L.qtr));
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_core_mu(const tpp_ctx* c, cudaStream_t s) {
  const int n = c->n, mu = c->mu, nn = n * n, m = 2 * mu + 2, p = (nn < m) ? nn : m;
  const size_t smem = (size_t)(m * m + m * p) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_core_mu, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_core_mu<<<(unsigned)c->E, 128, smem, s>>>(n, mu, c->E, c->prob.h, c->p<MuTables>(c->L.mutab),
                                              c->p<double>(c->L.cx), c->p<double>(c->L.cy),
                                              c->p<double>(c->L.fa), c->p<double>(c->L.rb),
                                              c->p<double>(c->L.kco),
                                              c->curved ? c->p<double>(c->L.mq) : nullptr);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_traces_mu(const tpp_ctx* c, const double* x, double* tr, cudaStream_t s,
                             const int32_t* skip) {
  k_traces_mu<double><<<152 * 8, 256, 0, s>>>(c->p<Tables>(c->L.tables), c->p<MuTables>(c->L.mutab),
                                              c->n, c->mu, c->EB, x, tr, skip);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_traces_mu_f32(const tpp_ctx* c, const float* x, float* tr, cudaStream_t s,
                                 const int32_t* skip) {
  k_traces_mu<float><<<152 * 8, 256, 0, s>>>(c->p<Tables>(c->L.tables), c->p<MuTables>(c->L.mutab),
                                             c->n, c->mu, c->EB, x, tr, skip);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_dg_apply_mu(const tpp_ctx* c, const double* x, const double* tr, double* y,
                               const int32_t* skip, cudaStream_t s, double mass) {
  return dg_apply_mu_t<double>(c, c->p<double>(c->L.cx), c->p<double>(c->L.cy),
                               c->p<double>(c->L.fa), x, tr, y, skip, s, mass,
                               c->curved ? c->p<double>(c->L.mq) : nullptr);
}

cudaError_t launch_dg_apply_mu_f32(const tpp_ctx* c, const float* x, const float* tr, float* y,
                                   const int32_t* skip, cudaStream_t s) {
  const float* f = c->p<float>(c->L.opf);
  const OpF32Layout O = op_f32_layout(c);
  return dg_apply_mu_t<float>(c, f + O.cx, f + O.cy, f + O.fa, x, tr, y, skip, s, 1.0,
                              c->curved ? f + O.mq : nullptr);
}

}  // namespace tpp
