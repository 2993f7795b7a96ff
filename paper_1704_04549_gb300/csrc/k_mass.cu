// Element-wise inversion of the exact mass matrix (Sec. 3.3): every element's
//   M_K = (G^T W (x) ... (x) G^T W) J_T (G (x) ... (x) G)
// with a mu-point Gauss-Legendre rule (mu >= n; G the mu x n evaluation matrix of
// the nodal basis at those points, J_T the caller's |Jacobian determinant| there),
// solved by preconditioned conjugate gradients whose preconditioner is the
// under-integrated (n-point, collocated) mass matrix: diagonal, w (x) ... (x) w
// times J_T at the nodes.  Both operations cost O(p^(d+1)) per element by their
// tensor-product structure.  One CTA per (element, right-hand side) block, the
// vectors in shared memory, the matvec by 2d one-dimensional contractions.
#include <cmath>
#include <string>

#include "tpp_internal.cuh"

namespace tpp {

namespace {

// rule and interpolation matrix of the mass solve: xq[mu], wq[mu], G[a * n + j] =
// phi_j(xq_a) by the barycentric formula on the n nodes (phi_j = delta at a node)
__global__ void k_mass_tables(const Tables* T, int n, int mu, double* tab) {
  __shared__ double lam[TPP_MAX_N];
  double* xq = tab;
  double* wq = tab + TPP_MAX_MU;
  double* G = tab + 2 * TPP_MAX_MU;
  const int t = threadIdx.x;
  if (t < mu) gauss_legendre_node(mu, t, &xq[t], &wq[t]);
  if (t < n) {
    double prod = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != t) prod *= (T->x[t] - T->x[m]);
    lam[t] = 1.0 / prod;
  }
  __syncthreads();
  if (t < mu) {
    const double xi = xq[t];
    int hit = -1;
    double sum = 0.0;
    for (int m = 0; m < n; ++m) {
      if (xi == T->x[m]) hit = m;
      else sum += lam[m] / (xi - T->x[m]);
    }
    for (int j = 0; j < n; ++j)
      G[t * n + j] = (hit >= 0) ? (j == hit ? 1.0 : 0.0) : (lam[j] / (xi - T->x[j])) / sum;
  }
}

// y = M_K x for one element (all arrays in shared memory; jq: J_T at the mu^d points)
template <int DIM>
__device__ void mass_matvec(int n, int mu, const double* G, const double* wq,
                            const double* __restrict__ jq, const double* x, double* y, double* A,
                            double* B) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (DIM == 2) {
    // A[i + n b] = sum_j G[b][j] x[i + n j]
    for (int q = tid; q < n * mu; q += nt) {
      const int i = q % n, b = q / n;
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += G[b * n + j] * x[i + n * j];
      A[q] = s;
    }
    __syncthreads();
    // B[a + mu b] = w_a w_b J(a, b) sum_i G[a][i] A[i + n b]
    for (int q = tid; q < mu * mu; q += nt) {
      const int a = q % mu, b = q / mu;
      double s = 0.0;
      for (int i = 0; i < n; ++i) s += G[a * n + i] * A[i + n * b];
      B[q] = s * wq[a] * wq[b] * jq[q];
    }
    __syncthreads();
    // A[i + n b] = sum_a G[a][i] B[a + mu b]
    for (int q = tid; q < n * mu; q += nt) {
      const int i = q % n, b = q / n;
      double s = 0.0;
      for (int a = 0; a < mu; ++a) s += G[a * n + i] * B[a + mu * b];
      A[q] = s;
    }
    __syncthreads();
    // y[i + n j] = sum_b G[b][j] A[i + n b]
    for (int q = tid; q < n * n; q += nt) {
      const int i = q % n, j = q / n;
      double s = 0.0;
      for (int b = 0; b < mu; ++b) s += G[b * n + j] * A[i + n * b];
      y[q] = s;
    }
  } else {
    const int nn = n * n;
    // A[i + n j + n^2 c] = sum_k G[c][k] x[i + n j + n^2 k]
    for (int q = tid; q < nn * mu; q += nt) {
      const int ij = q % nn, c = q / nn;
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += G[c * n + k] * x[ij + nn * k];
      A[q] = s;
    }
    __syncthreads();
    // B[i + n b + n mu c] = sum_j G[b][j] A[i + n j + n^2 c]
    for (int q = tid; q < n * mu * mu; q += nt) {
      const int i = q % n, b = (q / n) % mu, c = q / (n * mu);
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += G[b * n + j] * A[i + n * j + nn * c];
      B[q] = s;
    }
    __syncthreads();
    // A[a + mu b + mu^2 c] = w_a w_b w_c J sum_i G[a][i] B[i + n b + n mu c]
    for (int q = tid; q < mu * mu * mu; q += nt) {
      const int a = q % mu, b = (q / mu) % mu, c = q / (mu * mu);
      double s = 0.0;
      for (int i = 0; i < n; ++i) s += G[a * n + i] * B[i + n * b + n * mu * c];
      A[q] = s * wq[a] * wq[b] * wq[c] * jq[q];
    }
    __syncthreads();
    // B[i + n b + n mu c] = sum_a G[a][i] A[a + mu b + mu^2 c]
    for (int q = tid; q < n * mu * mu; q += nt) {
      const int i = q % n, b = (q / n) % mu, c = q / (n * mu);
      double s = 0.0;
      for (int a = 0; a < mu; ++a) s += G[a * n + i] * A[a + mu * b + mu * mu * c];
      B[q] = s;
    }
    __syncthreads();
    // A[i + n j + n^2 c] = sum_b G[b][j] B[i + n b + n mu c]
    for (int q = tid; q < nn * mu; q += nt) {
      const int i = q % n, j = (q / n) % n, c = q / nn;
      double s = 0.0;
      for (int b = 0; b < mu; ++b) s += G[b * n + j] * B[i + n * b + n * mu * c];
      A[q] = s;
    }
    __syncthreads();
    // y[i + n j + n^2 k] = sum_c G[c][k] A[i + n j + n^2 c]
    for (int q = tid; q < nn * n; q += nt) {
      const int ij = q % nn, k = q / nn;
      double s = 0.0;
      for (int c = 0; c < mu; ++c) s += G[c * n + k] * A[ij + nn * c];
      y[q] = s;
    }
  }
  __syncthreads();
}

// PCG on M_K x = r from x = 0 for vector block blockIdx.x (element blk / R)
template <int DIM>
__global__ void __launch_bounds__(256)
k_mass_pcg(const Tables* T, const double* __restrict__ tab, int n, int mu, int R,
           const double* __restrict__ jq_all, const double* __restrict__ jn_all,
           const double* __restrict__ rhs, double* __restrict__ xout, double rtol, int max_iters,
           int32_t* iters, DevStatus* st) {
  extern __shared__ double sm[];
  __shared__ double red[8];
  const int nloc = (DIM == 2) ? n * n : n * n * n;
  const int nq = (DIM == 2) ? mu * mu : mu * mu * mu;
  const int nA = nq, nB = (DIM == 2) ? mu * mu : n * mu * mu;
  const int64_t blk = blockIdx.x, e = blk / R;
  double* G = sm;                 // mu n
  double* wq = G + mu * n;        // mu
  double* x = wq + mu;
  double* r = x + nloc;
  double* z = r + nloc;
  double* p = z + nloc;
  double* q = p + nloc;
  double* pinv = q + nloc;        // 1 / (under-integrated mass)
  double* A = pinv + nloc;
  double* B = A + nA;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int t = tid; t < mu * n; t += nt) G[t] = tab[2 * TPP_MAX_MU + t];
  for (int t = tid; t < mu; t += nt) wq[t] = tab[TPP_MAX_MU + t];
  const double* jq = jq_all + e * nq;
  const double* jn = jn_all + e * nloc;
  const double* b = rhs + blk * nloc;
  double bb = 0.0;
  for (int t = tid; t < nloc; t += nt) {
    const int i = t % n, j = (t / n) % n, k = t / (n * n);
    double wn = T->w[i] * T->w[j];
    if (DIM == 3) wn *= T->w[k];
    pinv[t] = 1.0 / (wn * jn[t]);
    const double bv = b[t];
    x[t] = 0.0;
    r[t] = bv;
    z[t] = bv * pinv[t];
    p[t] = z[t];
    bb += bv * bv;
  }
  const double bnorm = sqrt(block_sum(bb, red));
  double rz = 0.0;
  for (int t = tid; t < nloc; t += nt) rz += r[t] * z[t];
  rz = block_sum(rz, red);
  double rnorm = bnorm;
  int it = 0;
  while (rnorm > rtol * bnorm && it < max_iters) {
    mass_matvec<DIM>(n, mu, G, wq, jq, p, q, A, B);
    double pq = 0.0;
    for (int t = tid; t < nloc; t += nt) pq += p[t] * q[t];
    pq = block_sum(pq, red);
    const double alpha = rz / pq;
    double rr = 0.0;
    for (int t = tid; t < nloc; t += nt) {
      x[t] += alpha * p[t];
      r[t] -= alpha * q[t];
      rr += r[t] * r[t];
    }
    rnorm = sqrt(block_sum(rr, red));
    ++it;
    double rz_new = 0.0;
    for (int t = tid; t < nloc; t += nt) {
      z[t] = r[t] * pinv[t];
      rz_new += r[t] * z[t];
    }
    rz_new = block_sum(rz_new, red);
    const double beta = rz_new / rz;
    rz = rz_new;
    for (int t = tid; t < nloc; t += nt) p[t] = z[t] + beta * p[t];
    __syncthreads();
  }
  for (int t = tid; t < nloc; t += nt) xout[blk * nloc + t] = x[t];
  if (tid == 0) {
    if (iters) iters[blk] = it;
    if (rnorm > rtol * bnorm) atomicAdd(&st->mass_unconverged, 1);
  }
}

size_t mass_smem(int dim, int n, int mu) {
  const size_t nloc = (dim == 2) ? (size_t)n * n : (size_t)n * n * n;
  const size_t nA = (dim == 2) ? (size_t)mu * mu : (size_t)mu * mu * mu;
  const size_t nB = (dim == 2) ? (size_t)mu * mu : (size_t)n * mu * mu;
  return ((size_t)mu * n + mu + 6 * nloc + nA + nB) * sizeof(double);
}

}  // namespace
}  // namespace tpp

using namespace tpp;

extern "C" tpp_status tpp_mass_solve(const tpp_ctx* c, int32_t mu, const double* jac_q,
                                     const double* jac_n, const double* r, double* x,
                                     int32_t nrhs, double rtol, int32_t max_iters, int32_t* iters,
                                     void* stream) {
  if (!c || !jac_q || !jac_n || !r || !x || r == x) {
    set_error("tpp_mass_solve: context, Jacobians, r and x non-NULL, r != x");
    return TPP_ERR_INVALID_ARG;
  }
  if (mu < c->n || mu > TPP_MAX_MU || nrhs < 1 || nrhs > c->R || !(rtol > 0.0) ||
      max_iters < 1) {
    set_error("tpp_mass_solve: n <= mu <= 64, 1 <= nrhs <= the problem's nrhs, rtol > 0, "
              "max_iters >= 1");
    return TPP_ERR_INVALID_ARG;
  }
  const size_t smem = mass_smem(c->dim, c->n, mu);
  if (smem > 200 * 1024) {
    set_error("tpp_mass_solve: n = " + std::to_string(c->n) + ", mu = " + std::to_string(mu) +
              " needs " + std::to_string(smem) + " bytes of shared memory per element (limit "
              "204800)");
    return TPP_ERR_UNSUPPORTED;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevStatus* st = c->p<DevStatus>(c->L.status);
  double* tab = c->p<double>(c->L.mtab);
  {
    cudaError_t e = cudaMemsetAsync(&st->mass_unconverged, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return cuda_check(e, "reset status");
    k_mass_tables<<<1, 64, 0, s>>>(c->p<Tables>(c->L.tables), c->n, mu, tab);
    count_launch();
    const unsigned blocks = (unsigned)(c->E * nrhs);
    if (c->dim == 2) {
      e = cudaFuncSetAttribute(k_mass_pcg<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e == cudaSuccess)
        k_mass_pcg<2><<<blocks, 256, smem, s>>>(c->p<Tables>(c->L.tables), tab, c->n, mu, nrhs,
                                               jac_q, jac_n, r, x, rtol, max_iters, iters, st);
    } else {
      e = cudaFuncSetAttribute(k_mass_pcg<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e == cudaSuccess)
        k_mass_pcg<3><<<blocks, 256, smem, s>>>(c->p<Tables>(c->L.tables), tab, c->n, mu, nrhs,
                                               jac_q, jac_n, r, x, rtol, max_iters, iters, st);
    }
    count_launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(e, "k_mass_pcg");
    int32_t bad = 0;
    e = cudaMemcpyAsync(&bad, &st->mass_unconverged, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_check(e, "tpp_mass_solve sync");
    if (bad) {
      set_error(std::to_string(bad) + " element mass solve(s) hit max_iters");
      return TPP_ERR_NOT_CONVERGED;
    }
  }
  return TPP_OK;
}
