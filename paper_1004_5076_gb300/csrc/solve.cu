// Right-hand side, GMRES with FP64 Arnoldi and iterative refinement, fields
// at interior points and the reflection fit.
//
// * rhs: tested incident field b (Appendix A): per row type <X, E_inc>,
//   <X, H_inc>, <X, H_inc> (Eq. 13), <sigma X, E_inc> (Eq. 14) for an
//   interior source (Eqs. 8-9); the mirrored combination, with
//   <sigma n x X, E_inc> in Eq. 13, for an exterior source.
// * solve: restarted GMRES (the paper's iterative solver, Appendix B) with
//   classical Gram-Schmidt applied twice in FP64 on the device; Hessenberg
//   least squares by Givens rotations; right-preconditioned by the inverse
//   per-edge diagonal blocks (the block-diagonal preconditioner of
//   Appendix B).  In complex64 mode the Krylov vectors stay FP64 and only
//   the operator runs in complex64.  An outer FP64 residual r = b - A x
//   drives iterative refinement in both modes.
// * fields / reflection: total interior field E_inc + E_i(J_i, M_i) (Eq. 8) at
//   probe points by the triangle quadrature, and a least-squares split of the
//   on-axis field into forward and backward waves (Table 1's reflection).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

template <typename R>
int compute_summ(scabem_op* op, const cx<R>* x, cx<R>* summ, cudaStream_t s);

namespace {

using cd = cx<double>;

__device__ __forceinline__ cd cexpd(cd z) {
  double s, c;
  sincos(z.im, &s, &c);
  const double e = exp(z.re);
  return mk(e * c, e * s);
}
__device__ __forceinline__ cd cdivd(cd a, cd b) {
  const double d = b.re * b.re + b.im * b.im;
  return mk((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
__device__ __forceinline__ cd csqrtd(cd z) {
  const double r = hypot(z.re, z.im);
  if (r == 0.0) return mk(0.0, 0.0);
  const double s = sqrt(0.5 * (r + fabs(z.re)));
  if (z.re >= 0.0) return mk(s, z.im / (2.0 * s));
  return mk(fabs(z.im) / (2.0 * s), copysign(s, z.im));
}

// Incident E and H (eta0 = 1 units) of source S in a medium (k, z).
__device__ void incident(const scabem_source& S, double k, double z, const double* r, cd* E, cd* H) {
  if (S.kind == 0) {
    const double ph = k * (S.dir[0] * r[0] + S.dir[1] * r[1] + S.dir[2] * r[2]);
    double sn, cs;
    sincos(ph, &sn, &cs);
    const cd e = mk(cs, -sn);
    const double dxp[3] = {S.dir[1] * S.pol[2] - S.dir[2] * S.pol[1], S.dir[2] * S.pol[0] - S.dir[0] * S.pol[2],
                           S.dir[0] * S.pol[1] - S.dir[1] * S.pol[0]};
    for (int c = 0; c < 3; ++c) {
      E[c] = S.pol[c] * e;
      H[c] = (dxp[c] / z) * e;
    }
    return;
  }
  const double b = S.kind == 2 ? S.b : 0.0;
  cd D[3];
  for (int c = 0; c < 3; ++c) D[c] = mk(r[c] - S.pos[c], b * S.dir[c]);  // r - (pos - j b dir)
  const cd R2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
  const cd R = csqrtd(R2);
  const cd iR = cdivd(mk(1.0, 0.0), R);
  cd Rh[3];
  for (int c = 0; c < 3; ++c) Rh[c] = D[c] * iR;
  const cd G = (1.0 / (4.0 * M_PI)) * (cexpd(mk(0.0, -k) * R) * iR);
  const cd u = mk(0.0, k) + iR;
  const cd G1 = -(u * G);
  const cd G2 = (u * u + iR * iR) * G;
  const cd rp = S.pol[0] * Rh[0] + S.pol[1] * Rh[1] + S.pol[2] * Rh[2];
  const cd G1R = G1 * iR;
  for (int c = 0; c < 3; ++c) {
    const cd hess = (G2 * rp) * Rh[c] + G1R * (mk(S.pol[c], 0.0) - rp * Rh[c]);
    const cd L = mk(0.0, k) * (S.pol[c] * G + (1.0 / (k * k)) * hess);
    E[c] = -z * L;
  }
  H[0] = G1 * (Rh[1] * S.pol[2] - Rh[2] * S.pol[1]);
  H[1] = G1 * (Rh[2] * S.pol[0] - Rh[0] * S.pol[2]);
  H[2] = G1 * (Rh[0] * S.pol[1] - Rh[1] * S.pol[0]);
}

__global__ void k_rhs(scabem_source S, const double* __restrict__ tri, const double* __restrict__ cX,
                      const double* __restrict__ qp, const double* __restrict__ qw, const double* __restrict__ sig,
                      int64_t nt, int q, double k, double z, cd* __restrict__ val) {
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= nt * 3) return;
  const int64_t t = gid / 3;
  const int kk = (int)(gid - t * 3);
  const double* g = tri + 16 * t;
  const double cxk = cX[gid];
  cd tE = mk(0.0, 0.0), tH = tE, tnsE = tE, tsE = tE;
  for (int a = 0; a < q; ++a) {
    const int64_t Qa = t * q + a;
    const double r[3] = {qp[3 * Qa], qp[3 * Qa + 1], qp[3 * Qa + 2]};
    cd E[3], H[3];
    incident(S, k, z, r, E, H);
    double X[3];
    for (int c = 0; c < 3; ++c) X[c] = cxk * (r[c] - g[3 * kk + c]);
    const double* n = g + 12;
    const double nX[3] = {n[1] * X[2] - n[2] * X[1], n[2] * X[0] - n[0] * X[2], n[0] * X[1] - n[1] * X[0]};
    const double w = qw[Qa];
    const cd xe = X[0] * E[0] + X[1] * E[1] + X[2] * E[2];
    tE += w * xe;
    tH += w * (X[0] * H[0] + X[1] * H[1] + X[2] * H[2]);
    tnsE += (w * sig[Qa]) * (nX[0] * E[0] + nX[1] * E[1] + nX[2] * E[2]);
    tsE += (w * sig[Qa]) * xe;
  }
  // rows: <X,E>, <X,H>, Eq. 13 (<X,H> and <sigma n x X, E>), Eq. 14
  cd* o = val + gid * 4;
  if (S.side == 0) {
    o[0] = tE;
    o[1] = tH;
    o[2] = tH;
    o[3] = tsE;
  } else {
    o[0] = -tE;
    o[1] = -tH;
    o[2] = tnsE - tH;
    o[3] = mk(0.0, 0.0);
  }
}

// Right-hand-side part of the conductivity sensitivity, one thread per
// quadrature point: hs[p] -= eta0 sum_kk lam_row d(rhs_row)/d sg, the
// sigma-weighted incident-field terms of k_rhs (Eq. 14 rows for an interior
// source, Eq. 13 rows for an exterior one).
__global__ void k_rhs_sens(scabem_source S, const double* __restrict__ tri, const double* __restrict__ cX,
                           const double* __restrict__ qp, const double* __restrict__ qw, const int32_t* __restrict__ valrow,
                           const cd* __restrict__ lam, int64_t Q, int q, double k, double z, cd* __restrict__ hs) {
  const int64_t Qa = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (Qa >= Q) return;
  const int64_t t = Qa / q;
  const double* g = tri + 16 * t;
  const double r[3] = {qp[3 * Qa], qp[3 * Qa + 1], qp[3 * Qa + 2]};
  cd E[3], H[3];
  incident(S, k, z, r, E, H);
  const double w = qw[Qa];
  const double* n = g + 12;
  cd acc = mk(0.0, 0.0);
  for (int kk = 0; kk < 3; ++kk) {
    double X[3];
    for (int c = 0; c < 3; ++c) X[c] = cX[3 * t + kk] * (r[c] - g[3 * kk + c]);
    const int row = valrow[(t * 3 + kk) * 4 + (S.side == 0 ? 3 : 2)];
    if (row < 0) continue;
    cd d;
    if (S.side == 0) {
      d = X[0] * E[0] + X[1] * E[1] + X[2] * E[2];
    } else {
      const double nX[3] = {n[1] * X[2] - n[2] * X[1], n[2] * X[0] - n[0] * X[2], n[0] * X[1] - n[1] * X[0]};
      d = nX[0] * E[0] + nX[1] * E[1] + nX[2] * E[2];
    }
    acc += lam[row] * (w * d);
  }
  hs[Qa] -= ETA0 * acc;
}

// Gradient reductions over the quadrature points (one block per parameter,
// fixed tree order): g[i] = sum_p dsigma_p/dc_i hs[p].
constexpr int GRAD_THREADS = 256;
__device__ void block_sum_store(cd v, cd* out) {
  __shared__ double sr[GRAD_THREADS], si[GRAD_THREADS];
  sr[threadIdx.x] = v.re;
  si[threadIdx.x] = v.im;
  __syncthreads();
  for (int st = GRAD_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sr[threadIdx.x] += sr[threadIdx.x + st];
      si[threadIdx.x] += si[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = mk(sr[0], si[0]);
}

// B-spline coefficient i: dsigma_p/dc_i = N_i(s_p), by de Boor's scheme on
// the unit coefficient vector (the same knots as k_sigma_bspline).
__global__ void k_grad_bspline(const double* __restrict__ qp, int64_t Q, double x0, double L, int axis, int ncoef,
                               const cd* __restrict__ hs, cd* __restrict__ g) {
  const int ci = blockIdx.x;
  const int nspan = ncoef - 3;
  cd acc = mk(0.0, 0.0);
  for (int64_t p = threadIdx.x; p < Q; p += GRAD_THREADS) {
    const double s = (qp[3 * p + axis] - x0) / L;
    if (s < 0.0 || s > 1.0) continue;
    int j = (int)(s * nspan);
    if (j >= nspan) j = nspan - 1;
    if (ci < j || ci > j + 3) continue;  // N_i vanishes outside its four spans
    auto knot = [&](int m) {
      const int v = m - 3;
      return v <= 0 ? 0.0 : (v >= nspan ? 1.0 : (double)v / nspan);
    };
    const int sp = j + 3;
    double d[4];
    for (int r = 0; r < 4; ++r) d[r] = (sp - 3 + r == ci) ? 1.0 : 0.0;
    for (int lvl = 1; lvl <= 3; ++lvl)
      for (int r = 3; r >= lvl; --r) {
        const int m = sp - 3 + r;
        const double den = knot(m + 4 - lvl) - knot(m);
        const double al = den > 0.0 ? (s - knot(m)) / den : 0.0;
        d[r] = (1.0 - al) * d[r - 1] + al * d[r];
      }
    acc += d[3] * hs[p];
  }
  block_sum_store(acc, g + ci);
}

// Monomial segment i: dsigma_p/dsigma0_i = u(s_p)^d of that segment.
__global__ void k_grad_monomial(const double* __restrict__ qp, int64_t Q, const double* __restrict__ seg,
                                const cd* __restrict__ hs, cd* __restrict__ g) {
  const double* sg = seg + 6 * blockIdx.x;
  const int ax = (int)sg[4];
  cd acc = mk(0.0, 0.0);
  for (int64_t p = threadIdx.x; p < Q; p += GRAD_THREADS) {
    const double s = sg[5] * (qp[3 * p + ax] - sg[0]) / sg[1];
    if (s < 0.0) continue;
    acc += pow(s > 1.0 ? 1.0 : s, sg[3]) * hs[p];
  }
  block_sum_store(acc, g + blockIdx.x);
}

template <typename R>
__global__ void k_rows_out(const cd* __restrict__ val, const int32_t* __restrict__ rowsrc, int64_t N,
                           cx<R>* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const cd v = val[rowsrc[2 * i]] + val[rowsrc[2 * i + 1]];
  y[i] = mk((R)v.re, (R)v.im);
}

// ---------------------------------------------------------------- BLAS-1 style kernels (FP64)
constexpr int DOT_THREADS = 256;
constexpr int DOT_BLOCKS = 304;  // 2 x 152 SMs

// Tall-skinny dot products for the Arnoldi step: part[b * ldp + c] = sum
// over row block b of conj(V[:, c]) . w, for the tile of DOT_TC columns
// c0 = blockIdx.y * DOT_TC (w is read once per tile).
constexpr int DOT_TC = 8;
__global__ void __launch_bounds__(DOT_THREADS) k_dots(const cd* __restrict__ V, int64_t ldv, int nv,
                                                      const cd* __restrict__ w, int64_t N, cd* __restrict__ part,
                                                      int ldp) {
  __shared__ double sm[DOT_THREADS / 32][2 * DOT_TC];
  const int c0 = blockIdx.y * DOT_TC;
  const int nc = min(DOT_TC, nv - c0);
  double ar[DOT_TC], ai[DOT_TC];
#pragma unroll
  for (int c = 0; c < DOT_TC; ++c) ar[c] = ai[c] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const cd b = w[i];
#pragma unroll
    for (int c = 0; c < DOT_TC; ++c)
      if (c < nc) {
        const cd a = V[(int64_t)(c0 + c) * ldv + i];
        ar[c] += a.re * b.re + a.im * b.im;
        ai[c] += a.re * b.im - a.im * b.re;
      }
  }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < DOT_TC; ++c)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar[c] += __shfl_xor_sync(0xffffffffu, ar[c], o);
      ai[c] += __shfl_xor_sync(0xffffffffu, ai[c], o);
    }
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < DOT_TC; ++c) {
      sm[wp][2 * c] = ar[c];
      sm[wp][2 * c + 1] = ai[c];
    }
  __syncthreads();
  if (threadIdx.x < 2 * nc) {
    double v = 0.0;
    for (int k = 0; k < DOT_THREADS / 32; ++k) v += sm[k][threadIdx.x];
    double* o = reinterpret_cast<double*>(part + (int64_t)blockIdx.x * ldp + c0);
    o[threadIdx.x] = v;
  }
}

__global__ void k_reduce_parts(const cd* __restrict__ part, int nb, int nv, cd* __restrict__ out) {
  __shared__ double sre[DOT_THREADS], sim[DOT_THREADS];
  const int c = blockIdx.x;
  double ar = 0.0, ai = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    ar += part[(int64_t)b * nv + c].re;
    ai += part[(int64_t)b * nv + c].im;
  }
  sre[threadIdx.x] = ar;
  sim[threadIdx.x] = ai;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sre[threadIdx.x] += sre[threadIdx.x + st];
      sim[threadIdx.x] += sim[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = mk(sre[0], sim[0]);
}

// w -= V h, and nparts[b] = sum over block b's rows of |w|^2 (new w)
__global__ void __launch_bounds__(DOT_THREADS) k_vsub_norm(const cd* __restrict__ V, int64_t ldv, int nv,
                                                           const cd* __restrict__ h, cd* __restrict__ w, int64_t N,
                                                           double* __restrict__ nparts) {
  __shared__ double sm[DOT_THREADS / 32];
  double nn = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    cd acc = w[i];
    for (int c = 0; c < nv; ++c) {
      const cd a = V[(int64_t)c * ldv + i], b = h[c];
      acc.re -= a.re * b.re - a.im * b.im;
      acc.im -= a.re * b.im + a.im * b.re;
    }
    w[i] = acc;
    nn += acc.re * acc.re + acc.im * acc.im;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = nn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int k = 0; k < DOT_THREADS / 32; ++k) v += sm[k];
    nparts[blockIdx.x] = v;
  }
}

// out->re = sqrt(sum of nparts), out->im = 0 (one block)
__global__ void k_norm_fin(const double* __restrict__ nparts, int nb, cd* __restrict__ out) {
  __shared__ double sm[DOT_THREADS];
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v += nparts[b];
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = mk(sqrt(fmax(sm[0], 0.0)), 0.0);
}

// v = w / |w| with the norm read from the device (zero when it vanishes)
__global__ void k_scale_dev(const cd* __restrict__ w, const cd* __restrict__ nrm, cd* __restrict__ v, int64_t N) {
  const double n = nrm->re;
  const double s = n > 1e-300 ? 1.0 / n : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = s * w[i];
}

// w -= V h   (h on the device, nv entries)
__global__ void k_vsub(const cd* __restrict__ V, int64_t ldv, int nv, const cd* __restrict__ h, cd* __restrict__ w,
                       int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    cd acc = w[i];
    for (int c = 0; c < nv; ++c) {
      const cd a = V[(int64_t)c * ldv + i], b = h[c];
      acc.re -= a.re * b.re - a.im * b.im;
      acc.im -= a.re * b.im + a.im * b.re;
    }
    w[i] = acc;
  }
}

__global__ void k_scale_to(const cd* __restrict__ w, double s, cd* __restrict__ v, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = s * w[i];
}
__global__ void k_sub(const cd* __restrict__ a, const cd* __restrict__ b, cd* __restrict__ o, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = a[i] - b[i];
}
__global__ void k_add(cd* __restrict__ x, const cd* __restrict__ d, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += d[i];
}
__global__ void k_to_f(const cd* __restrict__ a, cx<float>* __restrict__ o, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = mk((float)a[i].re, (float)a[i].im);
}
__global__ void k_from_f(const cx<float>* __restrict__ a, cd* __restrict__ o, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = mk((double)a[i].re, (double)a[i].im);
}

struct Work {
  cd* V = nullptr;     // N x (m+1)
  cd* w = nullptr;     // N
  cd* t = nullptr;     // N
  cd* part = nullptr;  // DOT_BLOCKS x (m+1)
  cd* h = nullptr;     // 2 (m+1) + 1: both Gram-Schmidt passes' coefficients, then the norm
  double* nparts = nullptr;  // DOT_BLOCKS
  cd* z = nullptr;     // N, preconditioned Krylov vector
  cd* u = nullptr;     // N, solution in the preconditioned variables
  cx<float>* xf = nullptr;
  cx<float>* yf = nullptr;
  bool tr = false;  // solve with A^T
  ~Work() {
    cudaFree(z);
    cudaFree(u);
    cudaFree(V);
    cudaFree(w);
    cudaFree(t);
    cudaFree(part);
    cudaFree(h);
    cudaFree(nparts);
    cudaFree(xf);
    cudaFree(yf);
  }
};

// h_dev[c] = conj(V[:, c]) . w for c < nv, left on the device.  About
// DOT_BLOCKS blocks in all: row blocks x column tiles, so that each thread
// covers several rows before the block reduction.
int dots_dev(const cd* V, int64_t ldv, int nv, const cd* w, int64_t N, Work& W, cd* h_dev, cudaStream_t s) {
  const int tiles = (int)cdiv(nv, DOT_TC);
  int rb = DOT_BLOCKS / tiles;
  if (rb < 8) rb = 8;
  k_dots<<<dim3(rb, tiles), DOT_THREADS, 0, s>>>(V, ldv, nv, w, N, W.part, nv);
  CK(cudaGetLastError());
  k_reduce_parts<<<nv, DOT_THREADS, 0, s>>>(W.part, rb, nv, h_dev);
  CK(cudaGetLastError());
  return SCABEM_OK;
}

// out->re = |w| (device)
int norm_dev(const cd* w, int64_t N, Work& W, cd* out, cudaStream_t s) {
  k_vsub_norm<<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(nullptr, N, 0, nullptr, const_cast<cd*>(w), N, W.nparts);
  CK(cudaGetLastError());
  k_norm_fin<<<1, DOT_THREADS, 0, s>>>(W.nparts, DOT_BLOCKS, out);
  CK(cudaGetLastError());
  return SCABEM_OK;
}

int dots(const cd* V, int64_t ldv, int nv, const cd* w, int64_t N, Work& W, cudaStream_t s, std::vector<cd>& out) {
  int rc = dots_dev(V, ldv, nv, w, N, W, W.h, s);
  if (rc) return rc;
  out.resize(nv);
  CK(cudaMemcpyAsync(out.data(), W.h, sizeof(cd) * nv, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return SCABEM_OK;
}

int norm2(const cd* w, int64_t N, Work& W, cudaStream_t s, double& nrm) {
  std::vector<cd> d;
  int rc = dots(w, N, 1, w, N, W, s, d);
  if (rc) return rc;
  nrm = std::sqrt(std::max(d[0].re, 0.0));
  return SCABEM_OK;
}

// y = A v in FP64 storage, arithmetic in `prec`.
int op_apply64(scabem_op* op, const cd* v, cd* y, int prec, Work& W, cudaStream_t s) {
  const int64_t N = op->N;
  if (prec == SCABEM_C128) return W.tr ? apply_adjoint_one<double>(op, v, y, s) : apply_one<double>(op, v, y, s);
  k_to_f<<<DOT_BLOCKS, 256, 0, s>>>(v, W.xf, N);
  CK(cudaGetLastError());
  int rc = W.tr ? apply_adjoint_one<float>(op, W.xf, W.yf, s) : apply_one<float>(op, W.xf, W.yf, s);
  if (rc) return rc;
  k_from_f<<<DOT_BLOCKS, 256, 0, s>>>(W.yf, y, N);
  CK(cudaGetLastError());
  return SCABEM_OK;
}

// Restarted GMRES for A d = r from d = 0 (d, r on the device).  Returns the
// status and accumulates iterations.
int gmres(scabem_op* op, const cd* r, cd* d, int prec, double tol, int m, int maxit, Work& W, cudaStream_t s,
          int& iters, double& relres_est) {
  const int64_t N = op->N;
  CK(cudaMemsetAsync(d, 0, sizeof(cd) * N, s));
  CK(cudaMemsetAsync(W.u, 0, sizeof(cd) * N, s));
  double rn0;
  int rc = norm2(r, N, W, s, rn0);
  if (rc) return rc;
  if (!std::isfinite(rn0)) {
    set_error("non-finite right-hand side");
    return SCABEM_E_NONFINITE;
  }
  relres_est = 0.0;
  if (rn0 == 0.0) return SCABEM_OK;
  // working residual: t = r - A d (d accumulates over restarts)
  CK(cudaMemcpyAsync(W.t, r, sizeof(cd) * N, cudaMemcpyDeviceToDevice, s));
  std::vector<cd> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), hv, hv2, hbuf;
  double beta = rn0;
  while (true) {
    k_scale_to<<<DOT_BLOCKS, 256, 0, s>>>(W.t, 1.0 / beta, W.V, N);
    CK(cudaGetLastError());
    for (auto& z : g) z = mk(0.0, 0.0);
    g[0] = mk(beta, 0.0);
    int j = 0;
    bool done = false;
    for (; j < m && iters < maxit; ++j) {
      ++iters;
      // right preconditioning: w = A P^-1 v_j
      rc = precond_apply(op, W.V + (int64_t)j * N, W.z, s, W.tr);
      if (rc) return rc;
      rc = op_apply64(op, W.z, W.w, prec, W, s);
      if (rc) return rc;
      // classical Gram-Schmidt on the device, repeated only when the first
      // pass cancels most of w (|w'| < |w| / sqrt 2, the Daniel-Gragg-
      // Kaufman-Stewart test); the norms and coefficients come to the host
      // in one copy per pass, and the next basis vector is scaled on the device
      cd* h1 = W.h;
      cd* h2 = W.h + (m + 1);
      cd* hn0 = W.h + 2 * (m + 1);  // |w| before, after pass 1, after pass 2
      cd* hn1 = hn0 + 1;
      cd* hn2 = hn0 + 2;
      rc = norm_dev(W.w, N, W, hn0, s);
      if (rc) return rc;
      rc = dots_dev(W.V, N, j + 1, W.w, N, W, h1, s);
      if (rc) return rc;
      k_vsub_norm<<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(W.V, N, j + 1, h1, W.w, N, W.nparts);
      CK(cudaGetLastError());
      k_norm_fin<<<1, DOT_THREADS, 0, s>>>(W.nparts, DOT_BLOCKS, hn1);
      CK(cudaGetLastError());
      hbuf.resize(2 * (m + 1) + 3);
      CK(cudaMemcpyAsync(hbuf.data(), W.h, sizeof(cd) * (j + 1), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(hbuf.data() + 2 * (m + 1), hn0, sizeof(cd) * 2, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      hv.assign(hbuf.begin(), hbuf.begin() + j + 1);
      double hn = hbuf[2 * (m + 1) + 1].re;
      const cd* hnd = hn1;
      if (!(hn >= 0.70710678118654752 * hbuf[2 * (m + 1)].re)) {
        rc = dots_dev(W.V, N, j + 1, W.w, N, W, h2, s);
        if (rc) return rc;
        k_vsub_norm<<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(W.V, N, j + 1, h2, W.w, N, W.nparts);
        CK(cudaGetLastError());
        k_norm_fin<<<1, DOT_THREADS, 0, s>>>(W.nparts, DOT_BLOCKS, hn2);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(hbuf.data() + (m + 1), h2, sizeof(cd) * (j + 1), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hbuf.data() + 2 * (m + 1) + 2, hn2, sizeof(cd), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        hv2.assign(hbuf.begin() + (m + 1), hbuf.begin() + (m + 1) + j + 1);
        hn = hbuf[2 * (m + 1) + 2].re;
        hnd = hn2;
      } else {
        hv2.assign(j + 1, mk(0.0, 0.0));
      }
      if (j + 1 < m) {
        k_scale_dev<<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(W.w, hnd, W.V + (int64_t)(j + 1) * N, N);
        CK(cudaGetLastError());
      }
      if (!std::isfinite(hn)) {
        set_error("non-finite Krylov vector");
        return SCABEM_E_NONFINITE;
      }
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hv[i] + hv2[i];
      H[(size_t)(j + 1) * m + j] = mk(hn, 0.0);
      // apply previous rotations
      for (int i = 0; i < j; ++i) {
        const cd a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = conj(cs[i]) * a + conj(sn[i]) * b;
        H[(size_t)(i + 1) * m + j] = -(sn[i] * a) + cs[i] * b;
      }
      const cd a = H[(size_t)j * m + j];
      const double bre = hn;
      const double den = std::sqrt(a.re * a.re + a.im * a.im + bre * bre);
      if (den == 0.0) {
        set_error("GMRES breakdown");
        return SCABEM_E_BREAKDOWN;
      }
      cs[j] = mk(a.re / den, a.im / den);
      sn[j] = mk(bre / den, 0.0);
      H[(size_t)j * m + j] = mk(den, 0.0);
      H[(size_t)(j + 1) * m + j] = mk(0.0, 0.0);
      const cd gj = g[j];
      g[j] = conj(cs[j]) * gj;
      g[j + 1] = -(sn[j] * gj);
      relres_est = std::sqrt(g[j + 1].re * g[j + 1].re + g[j + 1].im * g[j + 1].im) / rn0;
      if (hn <= 1e-300 || relres_est <= tol) {
        ++j;
        done = true;
        break;
      }
    }
    // back substitution, d += V y
    std::vector<cd> y(j);
    for (int i = j - 1; i >= 0; --i) {
      cd acc = g[i];
      for (int l = i + 1; l < j; ++l) acc -= H[(size_t)i * m + l] * y[l];
      const cd hd = H[(size_t)i * m + i];
      const double dd = hd.re * hd.re + hd.im * hd.im;
      y[i] = mk((acc.re * hd.re + acc.im * hd.im) / dd, (acc.im * hd.re - acc.re * hd.im) / dd);
    }
    for (auto& z : y) z = -z;
    if (j > 0) {
      CK(cudaMemcpyAsync(W.h, y.data(), sizeof(cd) * j, cudaMemcpyHostToDevice, s));
      k_vsub<<<DOT_BLOCKS, 256, 0, s>>>(W.V, N, j, W.h, W.u, N);
      CK(cudaGetLastError());
    }
    rc = precond_apply(op, W.u, d, s, W.tr);  // d = P^-1 u
    if (rc) return rc;
    if (done || iters >= maxit) break;
    // true residual for the restart
    rc = op_apply64(op, d, W.w, prec, W, s);
    if (rc) return rc;
    k_sub<<<DOT_BLOCKS, 256, 0, s>>>(r, W.w, W.t, N);
    CK(cudaGetLastError());
    rc = norm2(W.t, N, W, s, beta);
    if (rc) return rc;
    relres_est = beta / rn0;
    if (relres_est <= tol) break;
  }
  return SCABEM_OK;
}

// ---------------------------------------------------------------- fields at points
// One block per (point, rhs): sum over all source quadrature points of the
// interior set: E = -z_i (jk A + (j/k) grad phi) - curl F_i, M_i = -M.
__global__ void k_fields(const cd* __restrict__ summ, const double* __restrict__ tri, const double* __restrict__ qp,
                         const double* __restrict__ qw, int64_t Q, int q, const double* __restrict__ pts, double k,
                         double z, scabem_source inc, int has_inc, cd* __restrict__ E) {
  const int pi = blockIdx.x;
  const double r[3] = {pts[3 * pi], pts[3 * pi + 1], pts[3 * pi + 2]};
  cd A[3], gp[3], cF[3];
  for (int c = 0; c < 3; ++c) A[c] = gp[c] = cF[c] = mk(0.0, 0.0);
  for (int64_t b = threadIdx.x; b < Q; b += blockDim.x) {
    const int64_t t = b / q;
    const double* g = tri + 16 * t;
    const double rel[3] = {qp[3 * b] - g[9], qp[3 * b + 1] - g[10], qp[3 * b + 2] - g[11]};
    const cd* si = summ + (3 * t + 1) * 4;
    const cd* sm = summ + (3 * t + 2) * 4;
    const double D[3] = {r[0] - qp[3 * b], r[1] - qp[3 * b + 1], r[2] - qp[3 * b + 2]};
    const double R = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    double sn, cs;
    sincos(k * R, &sn, &cs);
    const double w = qw[b] / (4.0 * M_PI * R);
    const cd G = mk(w * cs, -w * sn);
    const cd dG = -(mk(1.0 / R, k) * G) * (1.0 / R);  // times D gives grad G
    const cd rho = 2.0 * si[0];
    cd J[3], M[3];
    for (int c = 0; c < 3; ++c) {
      J[c] = rel[c] * si[0] - si[1 + c];
      M[c] = -(rel[c] * sm[0] - sm[1 + c]);
    }
    for (int c = 0; c < 3; ++c) {
      A[c] += G * J[c];
      gp[c] += (D[c] * dG) * rho;
    }
    const cd gx = D[0] * dG, gy = D[1] * dG, gz = D[2] * dG;
    cF[0] += gy * M[2] - gz * M[1];
    cF[1] += gz * M[0] - gx * M[2];
    cF[2] += gx * M[1] - gy * M[0];
  }
  __shared__ double red[256][2];
  cd* accs[9] = {&A[0], &A[1], &A[2], &gp[0], &gp[1], &gp[2], &cF[0], &cF[1], &cF[2]};
  cd tot[9];
  for (int v = 0; v < 9; ++v) {
    red[threadIdx.x][0] = accs[v]->re;
    red[threadIdx.x][1] = accs[v]->im;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) {
        red[threadIdx.x][0] += red[threadIdx.x + st][0];
        red[threadIdx.x][1] += red[threadIdx.x + st][1];
      }
      __syncthreads();
    }
    tot[v] = mk(red[0][0], red[0][1]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    cd Ei[3], Hi[3];
    for (int c = 0; c < 3; ++c) Ei[c] = mk(0.0, 0.0);
    if (has_inc) incident(inc, k, z, r, Ei, Hi);
    for (int c = 0; c < 3; ++c) {
      const cd jA = mk(-tot[c].im, tot[c].re), jg = mk(-tot[3 + c].im, tot[3 + c].re);
      E[3 * pi + c] = Ei[c] - z * (k * jA + (1.0 / k) * jg) - tot[6 + c];
    }
  }
}

// Least-squares split E(t) = a exp(-j beta t) + c exp(j beta t); one block,
// threads over beta candidates.  out: {Re r, Im r, beta, residual, SWR, r_swr}.
__global__ void k_fit(const cd* __restrict__ E, const double* __restrict__ tt, int npts, double blo, double bhi,
                      int nbeta, double* __restrict__ out) {
  __shared__ double best_res[256];
  __shared__ int best_i[256];
  double enorm = 0.0;
  for (int i = 0; i < npts; ++i) enorm += E[i].re * E[i].re + E[i].im * E[i].im;
  double bres = 1e300;
  int bi = -1;
  for (int ib = threadIdx.x; ib < nbeta; ib += blockDim.x) {
    const double beta = nbeta > 1 ? blo + (bhi - blo) * ib / (nbeta - 1) : blo;
    cd a12 = mk(0.0, 0.0), r1 = a12, r2 = a12;
    for (int i = 0; i < npts; ++i) {
      double sn, cs;
      sincos(beta * tt[i], &sn, &cs);
      const cd ep = mk(cs, sn);    // exp(+j beta t)
      const cd em = mk(cs, -sn);   // exp(-j beta t)
      a12 += ep * ep;              // conj(em) * ep
      r1 += ep * E[i];             // conj(em) * E
      r2 += em * E[i];             // conj(ep) * E
    }
    const double n = npts;
    const double det = n * n - (a12.re * a12.re + a12.im * a12.im);
    const cd a = (1.0 / det) * (n * r1 - a12 * r2);
    const cd c = (1.0 / det) * (n * r2 - conj(a12) * r1);
    double res = 0.0;
    for (int i = 0; i < npts; ++i) {
      double sn, cs;
      sincos(beta * tt[i], &sn, &cs);
      const cd f = a * mk(cs, -sn) + c * mk(cs, sn) - E[i];
      res += f.re * f.re + f.im * f.im;
    }
    if (res < bres) {
      bres = res;
      bi = ib;
    }
  }
  best_res[threadIdx.x] = bres;
  best_i[threadIdx.x] = bi;
  __syncthreads();
  if (threadIdx.x == 0) {
    int b = -1;
    double r = 1e300;
    for (int i = 0; i < blockDim.x; ++i)
      if (best_i[i] >= 0 && (best_res[i] < r || (best_res[i] == r && best_i[i] < b))) {
        r = best_res[i];
        b = best_i[i];
      }
    const double beta = nbeta > 1 ? blo + (bhi - blo) * b / (nbeta - 1) : blo;
    cd a12 = mk(0.0, 0.0), r1 = a12, r2 = a12;
    double emax = 0.0, emin = 1e300;
    for (int i = 0; i < npts; ++i) {
      double sn, cs;
      sincos(beta * tt[i], &sn, &cs);
      const cd ep = mk(cs, sn), em = mk(cs, -sn);
      a12 += ep * ep;
      r1 += ep * E[i];
      r2 += em * E[i];
      const double m = sqrt(E[i].re * E[i].re + E[i].im * E[i].im);
      emax = fmax(emax, m);
      emin = fmin(emin, m);
    }
    const double n = npts;
    const double det = n * n - (a12.re * a12.re + a12.im * a12.im);
    const cd a = (1.0 / det) * (n * r1 - a12 * r2);
    const cd c = (1.0 / det) * (n * r2 - conj(a12) * r1);
    const cd rr = cdivd(c, a);
    const double swr = emax / emin;
    out[0] = rr.re;
    out[1] = rr.im;
    out[2] = beta;
    out[3] = sqrt(r / enorm);
    out[4] = swr;
    out[5] = (swr - 1.0) / (swr + 1.0);
  }
}

// Decay-rate fit (Sec. III): least squares for E(t) = a exp(-g tau) +
// c exp(g tau), g = alpha + j beta, tau = t - tm with tm the midpoint of the
// samples (both waves decay along their direction of travel).  With
// phi1 = exp(-g tau), phi2 = exp(g tau) the normal equations are
//   [g11 g12; conj(g12) g22] [a; c] = [r1; r2],
//   g11 = sum exp(-2 alpha tau), g22 = sum exp(2 alpha tau),
//   g12 = sum exp(2 j beta tau), r1 = sum conj(phi1) E, r2 = sum conj(phi2) E.
// One block scans the nalpha x nbeta candidates (alpha-major), each with its
// explicit residual; the smallest wins, ties to the lowest index.
__device__ void decay_amplitudes(const cd* __restrict__ E, const double* __restrict__ tt, int npts, double tm,
                                 double al, double be, cd& a, cd& c) {
  double g11 = 0.0, g22 = 0.0;
  cd g12 = mk(0.0, 0.0), r1 = g12, r2 = g12;
  for (int i = 0; i < npts; ++i) {
    const double tau = tt[i] - tm;
    const double em = exp(-al * tau), ep = exp(al * tau);
    double sn, cs;
    sincos(be * tau, &sn, &cs);
    g11 += em * em;
    g22 += ep * ep;
    g12 += mk(cs * cs - sn * sn, 2.0 * sn * cs);
    r1 += mk(em * cs, em * sn) * E[i];   // conj(phi1) = exp(-alpha tau) exp(+j beta tau)
    r2 += mk(ep * cs, -ep * sn) * E[i];  // conj(phi2) = exp(alpha tau) exp(-j beta tau)
  }
  const double det = g11 * g22 - (g12.re * g12.re + g12.im * g12.im);
  a = (1.0 / det) * (g22 * r1 - g12 * r2);
  c = (1.0 / det) * (g11 * r2 - conj(g12) * r1);
}
__device__ double decay_residual(const cd* __restrict__ E, const double* __restrict__ tt, int npts, double tm,
                                 double al, double be, cd a, cd c) {
  double res = 0.0;
  for (int i = 0; i < npts; ++i) {
    const double tau = tt[i] - tm;
    const double em = exp(-al * tau), ep = exp(al * tau);
    double sn, cs;
    sincos(be * tau, &sn, &cs);
    const cd f = a * mk(em * cs, -em * sn) + c * mk(ep * cs, ep * sn) - E[i];
    res += f.re * f.re + f.im * f.im;
  }
  return res;
}
__global__ void k_fit_decay(const cd* __restrict__ E, const double* __restrict__ tt, int npts, double alo,
                            double ahi, int na, double blo, double bhi, int nb, double* __restrict__ out) {
  __shared__ double best_res[256];
  __shared__ int best_i[256];
  const double tm = 0.5 * (tt[0] + tt[npts - 1]);
  double enorm = 0.0;
  for (int i = 0; i < npts; ++i) enorm += E[i].re * E[i].re + E[i].im * E[i].im;
  const int ncand = na * nb;
  double bres = 1e300;
  int bi = -1;
  for (int ic = threadIdx.x; ic < ncand; ic += blockDim.x) {
    const int ia = ic / nb, ib = ic - (ic / nb) * nb;
    const double al = na > 1 ? alo + (ahi - alo) * ia / (na - 1) : alo;
    const double be = nb > 1 ? blo + (bhi - blo) * ib / (nb - 1) : blo;
    cd a, c;
    decay_amplitudes(E, tt, npts, tm, al, be, a, c);
    const double res = decay_residual(E, tt, npts, tm, al, be, a, c);
    if (res < bres) {
      bres = res;
      bi = ic;
    }
  }
  best_res[threadIdx.x] = bres;
  best_i[threadIdx.x] = bi;
  __syncthreads();
  if (threadIdx.x == 0) {
    int b = -1;
    double r = 1e300;
    for (int i = 0; i < blockDim.x; ++i)
      if (best_i[i] >= 0 && (best_res[i] < r || (best_res[i] == r && best_i[i] < b))) {
        r = best_res[i];
        b = best_i[i];
      }
    const int ia = b / nb, ib = b - (b / nb) * nb;
    const double al = na > 1 ? alo + (ahi - alo) * ia / (na - 1) : alo;
    const double be = nb > 1 ? blo + (bhi - blo) * ib / (nb - 1) : blo;
    cd a, c;
    decay_amplitudes(E, tt, npts, tm, al, be, a, c);
    const cd rr = cdivd(c, a);
    out[0] = al;
    out[1] = be;
    out[2] = sqrt(r / enorm);
    out[3] = rr.re;
    out[4] = rr.im;
    out[5] = sqrt(a.re * a.re + a.im * a.im);
  }
}

}  // namespace

int rhs_impl(scabem_op* op, const scabem_source* src, int nsrc, void* b, int64_t ld, int prec, cudaStream_t s) {
  cd* val = nullptr;
  CK(cudaMalloc(&val, sizeof(cd) * op->nt * 12));
  for (int i = 0; i < nsrc; ++i) {
    const scabem_source S = src[i];
    const double k = S.side == 0 ? op->ki : op->ke;
    const double z = S.side == 0 ? op->zi : op->ze;
    k_rhs<<<(int)cdiv(op->nt * 3, 128), 128, 0, s>>>(S, op->tri, op->cX, op->qp, op->qw, op->sig64, op->nt, op->q, k,
                                                     z, val);
    CK(cudaGetLastError());
    if (prec == SCABEM_C128)
      k_rows_out<double><<<(int)cdiv(op->N, 256), 256, 0, s>>>(val, op->rowsrc, op->N, (cd*)b + (int64_t)i * ld);
    else
      k_rows_out<float><<<(int)cdiv(op->N, 256), 256, 0, s>>>(val, op->rowsrc, op->N,
                                                              (cx<float>*)b + (int64_t)i * ld);
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(s));
  cudaFree(val);
  return SCABEM_OK;
}

// Gradient of lam^T (A x - b) with respect to the parameters of `basis`
// (x, lam: device complex128, N each).  g_out: host, 2 * entries doubles.
int sigma_gradient_impl(scabem_op* op, const cd* x, const cd* lam, const scabem_source* src, int nsrc,
                        const scabem_sigma* basis, double* g_out, cudaStream_t s) {
  const int64_t Q = op->Q, N = op->N;
  cd *hs = nullptr, *yscr = nullptr, *g = nullptr;
  double* dseg = nullptr;
  int64_t ng = basis->kind == SCABEM_SIGMA_PER_QPOINT ? Q
               : basis->kind == SCABEM_SIGMA_BSPLINE   ? basis->ncoef
                                                       : basis->nseg;
  int rc = SCABEM_OK;
  auto fail = [&](cudaError_t e, const char* what) { rc = cuda_fail(e, what); };
  cudaError_t e;
  if ((e = cudaMalloc(&hs, sizeof(cd) * Q)) != cudaSuccess) fail(e, "cudaMalloc");
  if (!rc && (e = cudaMalloc(&yscr, sizeof(cd) * N)) != cudaSuccess) fail(e, "cudaMalloc");
  if (!rc && (e = cudaMalloc(&g, sizeof(cd) * (ng > 0 ? ng : 1))) != cudaSuccess) fail(e, "cudaMalloc");
  if (!rc) rc = sigma_sensitivity_op(op, x, lam, hs, yscr, s);
  for (int i = 0; !rc && i < nsrc; ++i) {
    const double k = src[i].side == 0 ? op->ki : op->ke, z = src[i].side == 0 ? op->zi : op->ze;
    k_rhs_sens<<<(int)cdiv(Q, 256), 256, 0, s>>>(src[i], op->tri, op->cX, op->qp, op->qw, op->valrow, lam, Q,
                                                 op->q, k, z, hs);
    if ((e = cudaGetLastError()) != cudaSuccess) fail(e, "k_rhs_sens");
  }
  if (!rc && basis->kind == SCABEM_SIGMA_PER_QPOINT) {
    if ((e = cudaMemcpyAsync(g_out, hs, sizeof(cd) * Q, cudaMemcpyDeviceToHost, s)) != cudaSuccess) fail(e, "copy");
  } else if (!rc && basis->kind == SCABEM_SIGMA_BSPLINE) {
    k_grad_bspline<<<basis->ncoef, GRAD_THREADS, 0, s>>>(op->qp, Q, basis->x0, basis->L, basis->axis, basis->ncoef,
                                                         hs, g);
    if ((e = cudaGetLastError()) != cudaSuccess) fail(e, "k_grad_bspline");
    if (!rc && (e = cudaMemcpyAsync(g_out, g, sizeof(cd) * ng, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      fail(e, "copy");
  } else if (!rc && ng > 0) {
    if ((e = cudaMalloc(&dseg, sizeof(double) * 6 * ng)) != cudaSuccess) fail(e, "cudaMalloc");
    if (!rc && (e = cudaMemcpyAsync(dseg, basis->seg, sizeof(double) * 6 * ng, cudaMemcpyHostToDevice, s)) !=
                   cudaSuccess)
      fail(e, "copy");
    if (!rc) {
      k_grad_monomial<<<(int)ng, GRAD_THREADS, 0, s>>>(op->qp, Q, dseg, hs, g);
      if ((e = cudaGetLastError()) != cudaSuccess) fail(e, "k_grad_monomial");
    }
    if (!rc && (e = cudaMemcpyAsync(g_out, g, sizeof(cd) * ng, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      fail(e, "copy");
  }
  if (!rc && (e = cudaStreamSynchronize(s)) != cudaSuccess) fail(e, "cudaStreamSynchronize");
  cudaFree(hs);
  cudaFree(yscr);
  cudaFree(g);
  cudaFree(dseg);
  return rc;
}

int solve_impl(scabem_op* op, const void* bv, void* xv, int nrhs, int64_t ld, const scabem_solve_opts* o,
               cudaStream_t s, scabem_solve_info* info) {
  const int64_t N = op->N;
  const int m = o->restart;
  const int prec = o->prec;
  Work W;
  W.tr = o->transpose != 0;
  CK(cudaMalloc(&W.V, sizeof(cd) * N * (m + 1)));
  CK(cudaMalloc(&W.w, sizeof(cd) * N));
  CK(cudaMalloc(&W.t, sizeof(cd) * N));
  CK(cudaMalloc(&W.z, sizeof(cd) * N));
  CK(cudaMalloc(&W.u, sizeof(cd) * N));
  CK(cudaMalloc(&W.part, sizeof(cd) * DOT_BLOCKS * (m + 1)));
  CK(cudaMalloc(&W.h, sizeof(cd) * (2 * (m + 1) + 3)));
  CK(cudaMalloc(&W.nparts, sizeof(double) * DOT_BLOCKS));
  if (prec == SCABEM_C64) {
    CK(cudaMalloc(&W.xf, sizeof(cx<float>) * N));
    CK(cudaMalloc(&W.yf, sizeof(cx<float>) * N));
  }
  cd* r = nullptr;
  cd* d = nullptr;
  CK(cudaMalloc(&r, sizeof(cd) * N));
  CK(cudaMalloc(&d, sizeof(cd) * N));
  int status = SCABEM_OK;
  for (int col = 0; col < nrhs; ++col) {
    const cd* b = (const cd*)bv + (int64_t)col * ld;
    cd* x = (cd*)xv + (int64_t)col * ld;
    double bn;
    int rc = norm2(b, N, W, s, bn);
    if (rc) return rc;
    int iters = 0, refs = 0;
    double relres = 0.0;
    const int outer = o->max_refine > 0 ? o->max_refine : 1;
    const double tol_out = o->refine_tol > 0 ? o->refine_tol : o->tol;
    int st = SCABEM_E_NOCONV;
    for (int it = 0; it <= outer; ++it) {
      rc = W.tr ? apply_adjoint_one<double>(op, x, W.w, s) : apply_one<double>(op, x, W.w, s);
      if (rc) return rc;
      k_sub<<<DOT_BLOCKS, 256, 0, s>>>(b, W.w, r, N);
      CK(cudaGetLastError());
      double rn;
      rc = norm2(r, N, W, s, rn);
      if (rc) return rc;
      relres = bn > 0 ? rn / bn : 0.0;
      if (!std::isfinite(relres)) {
        st = SCABEM_E_NONFINITE;
        break;
      }
      if (relres <= tol_out) {
        st = SCABEM_OK;
        break;
      }
      if (it == outer || iters >= o->maxit) break;
      double est;
      rc = gmres(op, r, d, prec, o->tol, m, o->maxit, W, s, iters, est);
      if (rc) return rc;
      k_add<<<DOT_BLOCKS, 256, 0, s>>>(x, d, N);
      CK(cudaGetLastError());
      ++refs;
    }
    if (info) {
      info[col].iters = iters;
      info[col].refinements = refs;
      info[col].relres = relres;
      info[col].status = st;
    }
    if (st != SCABEM_OK && status == SCABEM_OK) status = st;
  }
  CK(cudaStreamSynchronize(s));
  cudaFree(r);
  cudaFree(d);
  if (status != SCABEM_OK) set_error("solver did not reach the requested residual");
  return status;
}

static int fields_dev(scabem_op* op, const cd* x, const double* dpts, int npts, const scabem_source* inc, cd* dE,
                      cudaStream_t s) {
  int rc = compute_summ<double>(op, x, op->d.summ, s);
  if (rc) return rc;
  scabem_source S{};
  if (inc) S = *inc;
  k_fields<<<npts, 256, 0, s>>>(op->d.summ, op->tri, op->qp, op->qw, op->Q, op->q, dpts, op->ki, op->zi, S,
                                inc ? 1 : 0, dE);
  CK(cudaGetLastError());
  return SCABEM_OK;
}

int fields_impl(scabem_op* op, const void* x, int nrhs, int64_t ld, const double* pts, int npts,
                const scabem_source* inc, double* E, cudaStream_t s) {
  double* dpts = nullptr;
  cd* dE = nullptr;
  CK(cudaMalloc(&dpts, sizeof(double) * 3 * npts));
  CK(cudaMalloc(&dE, sizeof(cd) * 3 * npts));
  CK(cudaMemcpyAsync(dpts, pts, sizeof(double) * 3 * npts, cudaMemcpyHostToDevice, s));
  for (int col = 0; col < nrhs; ++col) {
    int rc = fields_dev(op, (const cd*)x + (int64_t)col * ld, dpts, npts, inc, dE, s);
    if (rc) return rc;
    CK(cudaMemcpyAsync(E + (int64_t)col * 6 * npts, dE, sizeof(cd) * 3 * npts, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  cudaFree(dpts);
  cudaFree(dE);
  return SCABEM_OK;
}

int reflection_impl(scabem_op* op, const void* x, int nrhs, int64_t ld, const scabem_probe* pr,
                    const scabem_source* inc, double* out, cudaStream_t s) {
  const int npts = pr->npts;
  std::vector<double> pts(3 * npts), tt(npts);
  for (int i = 0; i < npts; ++i) {
    const double t = npts > 1 ? pr->t0 + (pr->t1 - pr->t0) * i / (npts - 1) : pr->t0;
    tt[i] = t;
    for (int c = 0; c < 3; ++c) pts[3 * i + c] = pr->p0[c] + (c == pr->axis ? t : 0.0);
  }
  double *dpts = nullptr, *dtt = nullptr, *dout = nullptr;
  cd *dE = nullptr, *dc = nullptr;
  CK(cudaMalloc(&dpts, sizeof(double) * 3 * npts));
  CK(cudaMalloc(&dtt, sizeof(double) * npts));
  CK(cudaMalloc(&dE, sizeof(cd) * 3 * npts));
  CK(cudaMalloc(&dc, sizeof(cd) * npts));
  CK(cudaMalloc(&dout, sizeof(double) * 6));
  CK(cudaMemcpyAsync(dpts, pts.data(), sizeof(double) * 3 * npts, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dtt, tt.data(), sizeof(double) * npts, cudaMemcpyHostToDevice, s));
  for (int col = 0; col < nrhs; ++col) {
    int rc = fields_dev(op, (const cd*)x + (int64_t)col * ld, dpts, npts, inc, dE, s);
    if (rc) return rc;
    CK(cudaMemcpy2DAsync(dc, sizeof(cd), (const char*)dE + sizeof(cd) * pr->comp, 3 * sizeof(cd), sizeof(cd), npts,
                         cudaMemcpyDeviceToDevice, s));
    k_fit<<<1, 256, 0, s>>>(dc, dtt, npts, pr->beta_lo, pr->beta_hi, pr->nbeta, dout);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out + 6 * col, dout, sizeof(double) * 6, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  cudaFree(dpts);
  cudaFree(dtt);
  cudaFree(dE);
  cudaFree(dc);
  cudaFree(dout);
  return SCABEM_OK;
}

// Decay-rate fit of given samples (host t, host complex128 E).
int decay_fit_impl(const double* t, const double* E, int npts, double alo, double ahi, int na, double blo, double bhi,
                   int nb, double* out, cudaStream_t s) {
  double *dt = nullptr, *dout = nullptr;
  cd* dE = nullptr;
  CK(cudaMalloc(&dt, sizeof(double) * npts));
  CK(cudaMalloc(&dE, sizeof(cd) * npts));
  CK(cudaMalloc(&dout, sizeof(double) * 6));
  CK(cudaMemcpyAsync(dt, t, sizeof(double) * npts, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dE, E, sizeof(cd) * npts, cudaMemcpyHostToDevice, s));
  k_fit_decay<<<1, 256, 0, s>>>(dE, dt, npts, alo, ahi, na, blo, bhi, nb, dout);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, dout, sizeof(double) * 6, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  cudaFree(dt);
  cudaFree(dE);
  cudaFree(dout);
  return SCABEM_OK;
}

// Decay rate along a probe line: the total interior field component there
// (as for the reflection), then the decay-rate fit.
int decay_rate_impl(scabem_op* op, const void* x, int nrhs, int64_t ld, const scabem_probe* pr, double alo,
                    double ahi, int na, const scabem_source* inc, double* out, cudaStream_t s) {
  const int npts = pr->npts;
  std::vector<double> pts(3 * npts), tt(npts);
  for (int i = 0; i < npts; ++i) {
    const double t = npts > 1 ? pr->t0 + (pr->t1 - pr->t0) * i / (npts - 1) : pr->t0;
    tt[i] = t;
    for (int c = 0; c < 3; ++c) pts[3 * i + c] = pr->p0[c] + (c == pr->axis ? t : 0.0);
  }
  double *dpts = nullptr, *dtt = nullptr, *dout = nullptr;
  cd *dE = nullptr, *dc = nullptr;
  CK(cudaMalloc(&dpts, sizeof(double) * 3 * npts));
  CK(cudaMalloc(&dtt, sizeof(double) * npts));
  CK(cudaMalloc(&dE, sizeof(cd) * 3 * npts));
  CK(cudaMalloc(&dc, sizeof(cd) * npts));
  CK(cudaMalloc(&dout, sizeof(double) * 6));
  CK(cudaMemcpyAsync(dpts, pts.data(), sizeof(double) * 3 * npts, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dtt, tt.data(), sizeof(double) * npts, cudaMemcpyHostToDevice, s));
  for (int col = 0; col < nrhs; ++col) {
    int rc = fields_dev(op, (const cd*)x + (int64_t)col * ld, dpts, npts, inc, dE, s);
    if (rc) return rc;
    CK(cudaMemcpy2DAsync(dc, sizeof(cd), (const char*)dE + sizeof(cd) * pr->comp, 3 * sizeof(cd), sizeof(cd), npts,
                         cudaMemcpyDeviceToDevice, s));
    k_fit_decay<<<1, 256, 0, s>>>(dc, dtt, npts, alo, ahi, na, pr->beta_lo, pr->beta_hi, pr->nbeta, dout);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out + 6 * col, dout, sizeof(double) * 6, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  cudaFree(dpts);
  cudaFree(dtt);
  cudaFree(dE);
  cudaFree(dc);
  cudaFree(dout);
  return SCABEM_OK;
}

// ---------------------------------------------------------------- right-hand side without allocation
// Some callers cannot allocate device memory while they run: code that lives
// inside another framework's memory pool (which has already reserved the
// device), real-time loops that cannot afford the device-wide
// synchronisation a cudaFree implies, and services that must not meet an
// out-of-memory error halfway through a run.  scabem_rhs allocates its
// per-call row-value scratch; scabem_rhs_noalloc runs the same two kernels
// with that scratch in the fixed device array below instead.
constexpr int64_t NOALLOC_MAX_TRIANGLES = 32768;
// nt * 3 local edges * 4 row types complex128 values: 6 MiB, held by every
// GPU that loads this library until the process exits.
static __device__ __align__(256) cd g_rhs_scratch[NOALLOC_MAX_TRIANGLES * 12];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 256;
std::mutex g_noalloc_mu;
cd* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the array's name is only a host-side stand-in in host code).
int noalloc_scratch(int dev, cd** out) {
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    set_error("scabem_rhs_noalloc: device ordinal out of range");
    return SCABEM_E_DEVICE;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rhs_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_rhs_scratch)");
    g_noalloc_ptr[dev] = static_cast<cd*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return SCABEM_OK;
}
}  // namespace

extern "C" int scabem_rhs_noalloc(scabem_op_t op, const scabem_source* src, int32_t nsrc, void* b, int64_t ld,
                                  int32_t prec, void* stream) {
  if (!op || !src || !b || nsrc < 0 || ld < op->N || (prec != SCABEM_C64 && prec != SCABEM_C128)) {
    set_error("scabem_rhs_noalloc: bad argument");
    return SCABEM_E_ARG;
  }
  if (op->nt > NOALLOC_MAX_TRIANGLES) {
    set_error("scabem_rhs_noalloc: mesh has " + std::to_string(op->nt) + " triangles; the fixed scratch holds at most " +
              std::to_string(NOALLOC_MAX_TRIANGLES) + " (use scabem_rhs)");
    return SCABEM_E_ARG;
  }
  for (int i = 0; i < nsrc; ++i)
    if (src[i].kind < 0 || src[i].kind > 2 || src[i].side < 0 || src[i].side > 1) {
      set_error("scabem_rhs_noalloc: source kind must be 0..2 and side 0..1");
      return SCABEM_E_ARG;
    }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev != op->device) {
    set_error("scabem_rhs_noalloc: the operator's device is not the current device");
    return SCABEM_E_ARG;
  }
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, b) != cudaSuccess ||
      (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    set_error("scabem_rhs_noalloc: b must be device memory (host buffers would need staging)");
    return SCABEM_E_ARG;
  }
  cd* val = nullptr;
  int rc = noalloc_scratch(dev, &val);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < nsrc; ++i) {
    const scabem_source S = src[i];
    const double k = S.side == 0 ? op->ki : op->ke;
    const double z = S.side == 0 ? op->zi : op->ze;
    // k_rhs writes all nt*12 entries that k_rows_out reads, so the previous
    // call's contents never leak into this one.
    k_rhs<<<(int)cdiv(op->nt * 3, 128), 128, 0, s>>>(S, op->tri, op->cX, op->qp, op->qw, op->sig64, op->nt, op->q, k,
                                                     z, val);
    CK(cudaGetLastError());
    if (prec == SCABEM_C128)
      k_rows_out<double><<<(int)cdiv(op->N, 256), 256, 0, s>>>(val, op->rowsrc, op->N, (cd*)b + (int64_t)i * ld);
    else
      k_rows_out<float><<<(int)cdiv(op->N, 256), 256, 0, s>>>(val, op->rowsrc, op->N,
                                                              (cx<float>*)b + (int64_t)i * ld);
    CK(cudaGetLastError());
  }
  return SCABEM_OK;
}
