// Exact block-Jacobi comparator (Sec. 5: "exact block Jacobi" preconditioner).
//
// Each diagonal block S_e (n^2 x n^2 in 2D, n^3 x n^3 in 3D) is assembled entry by entry from
// the precomputed flux Jacobians (Eq. jac-entries with collocated quadrature):
//   S[(i,j),(k,l)] = h^2 w_i w_j d_ik d_jl
//     + d_lj (D_ki cx_kj + l1_i l1_k max(an_+x,j, 0) + l0_i l0_k max(an_-x,j, 0))
//     + d_ki (D_lj cy_il + l1_j l1_l max(an_+y,i, 0) + l0_j l0_l max(an_-y,i, 0)),
// an the scaled outward normal velocity of each face (only its outflow part enters the
// diagonal block),
// then LU-factored with partial pivoting (one CTA per element, in place in the
// workspace).  The apply is a forward / backward substitution per element.
#include "tpp_internal.cuh"

namespace tpp {

__global__ void k_bj_assemble_2d(const Tables* T, int n, double h, const double* cx,
                                 const double* cy, const double* fa, double* LU,
                                 const double* mq) {
  const int nn = n * n;
  const int64_t e = blockIdx.x;
  const double* fe = fa + e * 4 * n;          // outward normal velocities, faces -x, +x, -y, +y
  double* A = LU + e * (int64_t)nn * nn;      // row-major nn x nn
  for (int q = threadIdx.x; q < nn * nn; q += blockDim.x) {
    const int row = q / nn, col = q % nn;
    const int i = row % n, j = row / n, k = col % n, l = col / n;
    double v = 0.0;
    if (i == k && j == l) v += mq ? mq[e * nn + row] : h * h * T->w[i] * T->w[j];
    if (l == j) {
      v += T->D[k * n + i] * cx[e * nn + k + n * j];
      v += T->l1[i] * T->l1[k] * fmax(fe[1 * n + j], 0.0);
      v += T->l0[i] * T->l0[k] * fmax(fe[0 * n + j], 0.0);
    }
    if (k == i) {
      v += T->D[l * n + j] * cy[e * nn + i + n * l];
      v += T->l1[j] * T->l1[l] * fmax(fe[3 * n + i], 0.0);
      v += T->l0[j] * T->l0[l] * fmax(fe[2 * n + i], 0.0);
    }
    A[q] = v;
  }
}

// The 3D block (n^3 x n^3, node i + n j + n^2 k), the same terms in three directions:
//   S[(i,j,k),(i',j',k')] = h^3 w_i w_j w_k d_ii' d_jj' d_kk'
//     + d_jj' d_kk' (D_i'i cx_i'jk + l1_i l1_i' max(an_+x,jk, 0) + l0_i l0_i' max(an_-x,jk, 0))
//     + d_ii' d_kk' (D_j'j cy_ij'k + l1_j l1_j' max(an_+y,ik, 0) + l0_j l0_j' max(an_-y,ik, 0))
//     + d_ii' d_jj' (D_k'k cz_ijk' + l1_k l1_k' max(an_+z,ij, 0) + l0_k l0_k' max(an_-z,ij, 0)).
__global__ void k_bj_assemble_3d(const Tables* T, int n, double h, const double* cx,
                                 const double* cy, const double* cz, const double* fa,
                                 double* LU) {
  const int nn = n * n, n3 = nn * n;
  const int64_t e = blockIdx.x;
  const double* fe = fa + e * 6 * nn;
  const double* ce[3] = {cx + e * n3, cy + e * n3, cz + e * n3};
  double* A = LU + e * (int64_t)n3 * n3;
  const double h3 = h * h * h;
  for (int64_t q = threadIdx.x; q < (int64_t)n3 * n3; q += blockDim.x) {
    const int row = (int)(q / n3), col = (int)(q % n3);
    const int r3[3] = {row % n, (row / n) % n, row / nn};
    const int c3[3] = {col % n, (col / n) % n, col / nn};
    double v = 0.0;
    if (row == col) v += h3 * T->w[r3[0]] * T->w[r3[1]] * T->w[r3[2]];
    for (int d = 0; d < 3; ++d) {
      const int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
      if (r3[o1] != c3[o1] || r3[o2] != c3[o2]) continue;
      const int a = r3[d], ap = c3[d];
      int node[3] = {r3[0], r3[1], r3[2]};
      node[d] = ap;                                   // the coefficient sits at the column node
      v += T->D[ap * n + a] * ce[d][node[0] + n * node[1] + nn * node[2]];
      // tangential index of the face points: the two other directions, lower first
      const int lo = (d == 0) ? 1 : 0, hi = (d == 2) ? 1 : 2;
      const int t = r3[lo] + n * r3[hi];
      v += T->l0[a] * T->l0[ap] * fmax(fe[(2 * d) * nn + t], 0.0);
      v += T->l1[a] * T->l1[ap] * fmax(fe[(2 * d + 1) * nn + t], 0.0);
    }
    A[q] = v;
  }
}

// In-place LU with partial pivoting of one nb x nb row-major block per CTA.
__global__ void k_bj_lu(int nb, double* LU, int32_t* piv) {
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int prow;
  const int64_t e = blockIdx.x;
  double* A = LU + e * (int64_t)nb * nb;
  int32_t* P = piv + e * (int64_t)nb;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < nb; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + tid; i < nb; i += blockDim.x) {
      const double v = fabs(A[(int64_t)i * nb + k]);
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { red_v[wid] = best; red_i[wid] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bv = red_v[0];
      int b = red_i[0];
      for (int w = 1; w < nw; ++w)
        if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < b)) { bv = red_v[w]; b = red_i[w]; }
      prow = b;
      P[k] = b;
    }
    __syncthreads();
    const int p = prow;
    if (p != k)
      for (int c = tid; c < nb; c += blockDim.x) {
        const double t = A[(int64_t)k * nb + c];
        A[(int64_t)k * nb + c] = A[(int64_t)p * nb + c];
        A[(int64_t)p * nb + c] = t;
      }
    __syncthreads();
    const double d = A[(int64_t)k * nb + k];
    const double inv = (d != 0.0) ? 1.0 / d : 0.0;
    for (int i = k + 1 + tid; i < nb; i += blockDim.x) A[(int64_t)i * nb + k] *= inv;
    __syncthreads();
    const int rem = nb - k - 1;
    for (int q = tid; q < rem * rem; q += blockDim.x) {
      const int i = k + 1 + q / rem, c = k + 1 + q % rem;
      A[(int64_t)i * nb + c] -= A[(int64_t)i * nb + k] * A[(int64_t)k * nb + c];
    }
    __syncthreads();
  }
}

__global__ void k_bj_solve(int nb, const double* LU, const int32_t* piv, const double* b,
                           double* x, const int32_t* skip, int R) {
  if (skip && *skip) return;
  extern __shared__ double ys[];
  const int64_t blk = blockIdx.x, e = blk / R;   // vector block: right-hand side blk % R
  const double* A = LU + e * (int64_t)nb * nb;
  const int32_t* P = piv + e * (int64_t)nb;
  const int tid = threadIdx.x;
  for (int i = tid; i < nb; i += blockDim.x) ys[i] = b[blk * nb + i];
  __syncthreads();
  if (tid == 0)
    for (int k = 0; k < nb; ++k)
      if (P[k] != k) { const double t = ys[k]; ys[k] = ys[P[k]]; ys[P[k]] = t; }
  __syncthreads();
  for (int k = 0; k < nb; ++k) {         // L y = P b (unit lower)
    const double yk = ys[k];
    for (int i = k + 1 + tid; i < nb; i += blockDim.x) ys[i] -= A[(int64_t)i * nb + k] * yk;
    __syncthreads();
  }
  for (int k = nb - 1; k >= 0; --k) {    // U x = y
    if (tid == 0) ys[k] /= A[(int64_t)k * nb + k];
    __syncthreads();
    const double xk = ys[k];
    for (int i = tid; i < k; i += blockDim.x) ys[i] -= A[(int64_t)i * nb + k] * xk;
    __syncthreads();
  }
  for (int i = tid; i < nb; i += blockDim.x) x[blk * nb + i] = ys[i];
}

cudaError_t launch_bj_build(const tpp_ctx* c, cudaStream_t s) {
  if (c->dim == 3) {
    k_bj_assemble_3d<<<(unsigned)c->E, 256, 0, s>>>(
        c->p<Tables>(c->L.tables), c->n, c->prob.h, c->p<double>(c->L.cx),
        c->p<double>(c->L.cy), c->p<double>(c->L.cz), c->p<double>(c->L.fa),
        c->p<double>(c->L.bj_lu));
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_bj_lu<<<(unsigned)c->E, 256, 0, s>>>(c->nloc, c->p<double>(c->L.bj_lu),
                                           c->p<int32_t>(c->L.bj_piv));
    count_launch();
    return cudaGetLastError();
  }
  k_bj_assemble_2d<<<(unsigned)c->E, 256, 0, s>>>(
      c->p<Tables>(c->L.tables), c->n, c->prob.h, c->p<double>(c->L.cx), c->p<double>(c->L.cy),
      c->p<double>(c->L.fa), c->p<double>(c->L.bj_lu),
      c->curved ? c->p<double>(c->L.mq) : nullptr);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_bj_lu<<<(unsigned)c->E, 256, 0, s>>>(c->nloc, c->p<double>(c->L.bj_lu),
                                         c->p<int32_t>(c->L.bj_piv));
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_bj_apply(const tpp_ctx* c, const double* b, double* x, const int32_t* skip,
                            cudaStream_t s) {
  k_bj_solve<<<(unsigned)c->EB, 256, c->nloc * sizeof(double), s>>>(
      c->nloc, c->p<double>(c->L.bj_lu), c->p<int32_t>(c->L.bj_piv), b, x, skip, c->R);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_bj_lu(int nb, int64_t nblk, double* LU, int32_t* piv, cudaStream_t s) {
  k_bj_lu<<<(unsigned)nblk, 256, 0, s>>>(nb, LU, piv);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_bj_solve(int nb, int64_t nblk, int R, const double* LU, const int32_t* piv,
                            const double* b, double* x, const int32_t* skip, cudaStream_t s) {
  k_bj_solve<<<(unsigned)(nblk * R), 256, nb * sizeof(double), s>>>(nb, LU, piv, b, x, skip, R);
  count_launch();
  return cudaGetLastError();
}

}  // namespace tpp
