// The matvec y = A x of the grid-accelerated operator (one right-hand side).
//
//  K1 k_summ     RWG coefficients -> per-triangle current summaries
//                J(r) = a (r - c_t) - beta for the exterior J, interior J and
//                exterior M sets (current reduction, Eqs. 10-12)
//  K2 k_project  point sources at the quadrature points spread onto the grid
//                by the Lagrange stencils (12 fields)
//  K3-5          fft_conv (fft.cu): 12 -> 16 grid potentials (A, phi, F, psi
//                of each medium, Eqs. 15-16)
//  K6 k_interp   potentials, gradients and curls at the quadrature points
//  K7 k_near     near-field precorrection: exact minus grid panel moments
//  K8 k_test     Galerkin testing of Eqs. 1-3 (weak form), Eq. 13 and Eq. 14
//                (strong form, sigma-weighted, with the side-limit terms)
//     k_rows     per-edge sum of the two triangles' tested values
#include <cuda_runtime.h>

#include "common.cuh"

namespace {

template <typename R>
__device__ __forceinline__ cx<R> coef_of(const cx<R>* __restrict__ x, int32_t code) {
  if (code > 0) return x[code - 1];
  if (code < 0) return -x[-code - 1];
  return czero<R>();
}

// K1: one thread per triangle.  summ[(t*3+set)*4 + {a, bx, by, bz}]
template <typename R>
__global__ void k_summ(const cx<R>* __restrict__ x, const int32_t* __restrict__ unk, const double* __restrict__ cX,
                       const double* __restrict__ tri, int64_t nt, cx<R>* __restrict__ summ) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const double* g = tri + 16 * t;
  R rel[3][3];
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) rel[k][c] = (R)(g[3 * k + c] - g[9 + c]);
  R ck[3];
  for (int k = 0; k < 3; ++k) ck[k] = (R)cX[3 * t + k];
  for (int set = 0; set < 3; ++set) {
    cx<R> a = czero<R>(), b0 = a, b1 = a, b2 = a;
    for (int k = 0; k < 3; ++k) {
      const cx<R> j = ck[k] * coef_of(x, unk[(3 * t + k) * 3 + set]);
      a += j;
      b0 += rel[k][0] * j;
      b1 += rel[k][1] * j;
      b2 += rel[k][2] * j;
    }
    cx<R>* o = summ + (3 * t + set) * 4;
    o[0] = a;
    o[1] = b0;
    o[2] = b1;
    o[3] = b2;
  }
}

template <typename R>
__device__ __forceinline__ void atomic_add_cx(cx<R>* p, cx<R> v);
template <>
__device__ __forceinline__ void atomic_add_cx<float>(cx<float>* p, cx<float> v) {
  atomicAdd(reinterpret_cast<float2*>(p), make_float2(v.re, v.im));
}
template <>
__device__ __forceinline__ void atomic_add_cx<double>(cx<double>* p, cx<double> v) {
  atomicAdd(&p->re, v.re);
  atomicAdd(&p->im, v.im);
}

// K2: one thread per (quadrature point, stencil node).  Source fields
// [set*4 + {x, y, z, div}] of the exterior J, interior J and exterior M sets,
// each point source weighted by its quadrature weight.
template <typename R>
__global__ void k_project(const cx<R>* __restrict__ summ, const double* __restrict__ qp, const double* __restrict__ qw,
                          const double* __restrict__ tri, const int32_t* __restrict__ base, const R* __restrict__ L,
                          int64_t Q, int q, int p, int n0, int n1, int n2, cx<R>* __restrict__ grids) {
  const int p3 = p * p * p;
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= Q * p3) return;
  const int64_t Qi = gid / p3;
  const int sidx = (int)(gid - Qi * p3);
  const int i = sidx / (p * p), j = (sidx / p) % p, k = sidx % p;
  const int64_t t = Qi / q;
  const R W = L[(3 * Qi + 0) * p + i] * L[(3 * Qi + 1) * p + j] * L[(3 * Qi + 2) * p + k] * (R)qw[Qi];
  const double* g = tri + 16 * t;
  const R rel[3] = {(R)(qp[3 * Qi] - g[9]), (R)(qp[3 * Qi + 1] - g[10]), (R)(qp[3 * Qi + 2] - g[11])};
  const int64_t gi =
      ((int64_t)(base[3 * Qi] + i) * n1 + (base[3 * Qi + 1] + j)) * n2 + (base[3 * Qi + 2] + k);
  const int64_t ng = (int64_t)n0 * n1 * n2;
  for (int set = 0; set < 3; ++set) {
    const cx<R>* s = summ + (3 * t + set) * 4;
    const cx<R> a = s[0];
    for (int c = 0; c < 3; ++c) {
      const cx<R> J = rel[c] * a - s[1 + c];
      atomic_add_cx(grids + (set * 4 + c) * ng + gi, W * J);
    }
    atomic_add_cx(grids + (set * 4 + 3) * ng + gi, (R(2) * W) * a);
  }
}

// K6: one thread per (quadrature point, medium).  Output record (NREC):
// A(3) phi grad phi(3) curl A(3) F(3) psi grad psi(3) curl F(3).
template <typename R>
__global__ void k_interp(const cx<R>* __restrict__ grids, const int32_t* __restrict__ base, const R* __restrict__ L,
                         const R* __restrict__ dL, int64_t Q, int p, int n0, int n1, int n2, cx<R>* __restrict__ fpt) {
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= Q * 2) return;
  const int64_t Qi = gid >> 1;
  const int med = (int)(gid & 1);
  R Lx[MAXP], Ly[MAXP], Lz[MAXP], dx[MAXP], dy[MAXP], dz[MAXP];
  for (int i = 0; i < p; ++i) {
    Lx[i] = L[(3 * Qi + 0) * p + i];
    Ly[i] = L[(3 * Qi + 1) * p + i];
    Lz[i] = L[(3 * Qi + 2) * p + i];
    dx[i] = dL[(3 * Qi + 0) * p + i];
    dy[i] = dL[(3 * Qi + 1) * p + i];
    dz[i] = dL[(3 * Qi + 2) * p + i];
  }
  const int b0 = base[3 * Qi], b1 = base[3 * Qi + 1], b2 = base[3 * Qi + 2];
  const int64_t ng = (int64_t)n0 * n1 * n2;
  cx<R> v[8], gx[8], gy[8], gz[8];
  for (int f = 0; f < 8; ++f) v[f] = gx[f] = gy[f] = gz[f] = czero<R>();
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) {
      const R wxy = Lx[i] * Ly[j], dxy = dx[i] * Ly[j], xdy = Lx[i] * dy[j];
      const int64_t rowi = ((int64_t)(b0 + i) * n1 + (b1 + j)) * n2 + b2;
      for (int k = 0; k < p; ++k) {
        const R w = wxy * Lz[k], wx = dxy * Lz[k], wy = xdy * Lz[k], wz = wxy * dz[k];
        for (int f = 0; f < 8; ++f) {
          const cx<R> gv = grids[(med * 8 + f) * ng + rowi + k];
          axpy(v[f], w, gv);
          axpy(gx[f], wx, gv);
          axpy(gy[f], wy, gv);
          axpy(gz[f], wz, gv);
        }
      }
    }
  cx<R>* o = fpt + gid * NREC;
  for (int h = 0; h < 2; ++h) {
    const int f0 = 4 * h;  // A (h=0) or F (h=1)
    cx<R>* r = o + 10 * h;
    r[0] = v[f0];
    r[1] = v[f0 + 1];
    r[2] = v[f0 + 2];
    r[3] = v[f0 + 3];
    r[4] = gx[f0 + 3];
    r[5] = gy[f0 + 3];
    r[6] = gz[f0 + 3];
    r[7] = gy[f0 + 2] - gz[f0 + 1];
    r[8] = gz[f0 + 0] - gx[f0 + 2];
    r[9] = gx[f0 + 1] - gy[f0 + 0];
  }
}

// K7: one thread per (target point, medium).  Each near record (10 complex:
// dP0, dP1, dQ, dC) is loaded once and applied to the J and the M source of
// the pair; two pairs are kept in flight.
template <typename R>
__device__ __forceinline__ void near_accumulate(const cx<R>* d, const cx<R>* sj, const cx<R>* sm, R sgnm,
                                                cx<R>* accJ, cx<R>* accM) {
  const cx<R> d0 = d[0];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cx<R>* sv = h == 0 ? sj : sm;
    const R sg = h == 0 ? R(1) : sgnm;
    cx<R>* acc = h == 0 ? accJ : accM;
    const cx<R> al = sg * sv[0];
    const cx<R> be0 = sg * sv[1], be1 = sg * sv[2], be2 = sg * sv[3];
    const cx<R> be[3] = {be0, be1, be2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cfma(acc[c], al, d[1 + c]);
      acc[c] -= be[c] * d0;
      cfma(acc[4 + c], R(2) * al, d[4 + c]);
      cfma(acc[7 + c], al, d[7 + c]);
    }
    cfma(acc[3], R(2) * al, d0);
    acc[7] -= d[5] * be2 - d[6] * be1;  // - dQ x beta
    acc[8] -= d[6] * be0 - d[4] * be2;
    acc[9] -= d[4] * be1 - d[5] * be0;
  }
}

template <typename R>
__global__ void __launch_bounds__(128) k_near(const cx<R>* __restrict__ corr, const int32_t* __restrict__ noff,
                                              const int32_t* __restrict__ nsrc, const cx<R>* __restrict__ summ,
                                              int64_t Q, int q, cx<R>* __restrict__ fpt) {
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= Q * 2) return;
  const int64_t Qa = gid >> 1;
  const int med = (int)(gid & 1);
  const int64_t t = Qa / q;
  const int a = (int)(Qa - t * q);
  const R sgnm = med == 1 ? R(-1) : R(1);  // interior M = -M
  cx<R> accJ[NCORR], accM[NCORR];
  for (int c = 0; c < NCORR; ++c) accJ[c] = accM[c] = czero<R>();
  const int j0 = noff[t], j1 = noff[t + 1];
  const int64_t rec = (int64_t)q * 2 * NCORR;  // complex per pair
  const cx<R>* base = corr + ((int64_t)a * 2 + med) * NCORR;
  int j = j0;
  for (; j + 1 < j1; j += 2) {
    cx<R> dA[NCORR], dB[NCORR];
    const int64_t sA = nsrc[j], sB = nsrc[j + 1];
    const cx<R>* pA = base + (int64_t)j * rec;
    const cx<R>* pB = pA + rec;
#pragma unroll
    for (int c = 0; c < NCORR; ++c) {
      dA[c] = pA[c];
      dB[c] = pB[c];
    }
    near_accumulate(dA, summ + (3 * sA + med) * 4, summ + (3 * sA + 2) * 4, sgnm, accJ, accM);
    near_accumulate(dB, summ + (3 * sB + med) * 4, summ + (3 * sB + 2) * 4, sgnm, accJ, accM);
  }
  if (j < j1) {
    cx<R> dA[NCORR];
    const int64_t sA = nsrc[j];
    const cx<R>* pA = base + (int64_t)j * rec;
#pragma unroll
    for (int c = 0; c < NCORR; ++c) dA[c] = pA[c];
    near_accumulate(dA, summ + (3 * sA + med) * 4, summ + (3 * sA + 2) * 4, sgnm, accJ, accM);
  }
  cx<R>* o = fpt + gid * NREC;
  for (int c = 0; c < NCORR; ++c) {
    o[c] += accJ[c];
    o[10 + c] += accM[c];
  }
}

template <typename R>
__device__ __forceinline__ cx<R> dot3(const R* X, const cx<R>* V) {
  return X[0] * V[0] + X[1] * V[1] + X[2] * V[2];
}

// K8: one thread per (triangle, local edge k).  val[(t*3+k)*4 + type]:
// type 0 <X, E_e - E_i>, 1 <X, H_e - H_i> (weak forms); 2 Eq. 13, 3 Eq. 14.
template <typename R>
__global__ void k_test(const cx<R>* __restrict__ fpt, const cx<R>* __restrict__ summ, const double* __restrict__ tri,
                       const double* __restrict__ cX, const double* __restrict__ qp, const double* __restrict__ qw,
                       const R* __restrict__ sig, int64_t nt, int q, R ke, R ki, R ze, R zi,
                       cx<R>* __restrict__ val) {
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= nt * 3) return;
  const int64_t t = gid / 3;
  const int kk = (int)(gid - t * 3);
  const double* g = tri + 16 * t;
  const R cxk = (R)cX[gid];
  const R divX = R(2) * cxk;
  const R nrm[3] = {(R)g[12], (R)g[13], (R)g[14]};
  const cx<R>* se = summ + (3 * t + 0) * 4;
  const cx<R>* si = summ + (3 * t + 1) * 4;
  const cx<R>* sM = summ + (3 * t + 2) * 4;
  cx<R> v0 = czero<R>(), v1 = v0, v2 = v0, v3 = v0;
  const R kl[2] = {ke, ki}, zl[2] = {ze, zi};
  for (int a = 0; a < q; ++a) {
    const int64_t Qa = t * q + a;
    const R w = (R)qw[Qa];
    const R sg = sig[Qa];
    R X[3], rel[3];
    for (int c = 0; c < 3; ++c) {
      X[c] = cxk * (R)(qp[3 * Qa + c] - g[3 * kk + c]);
      rel[c] = (R)(qp[3 * Qa + c] - g[9 + c]);
    }
    cx<R> WE[3], WH[3], E[2][3];
    cx<R> wE = czero<R>(), wH = czero<R>();
    for (int c = 0; c < 3; ++c) WE[c] = WH[c] = czero<R>();
    for (int m = 0; m < 2; ++m) {
      const cx<R>* r = fpt + (Qa * 2 + m) * NREC;
      const R k = kl[m], z = zl[m];
      const R sgm = m == 0 ? R(1) : R(-1);
      const cx<R> phi = r[3], psi = r[13];
      wE += (sgm * z / k) * mulj(phi);
      wH += (sgm / (k * z)) * mulj(psi);
      for (int c = 0; c < 3; ++c) {
        const cx<R> A = r[c], gphi = r[4 + c], cA = r[7 + c], F = r[10 + c], cF = r[17 + c];
        const cx<R> jA = mulj(A), jF = mulj(F);
        WE[c] += sgm * ((-z * k) * jA - cF);
        WH[c] += sgm * (cA - (k / z) * jF);
        E[m][c] = -z * (k * jA + (R(1) / k) * mulj(gphi)) - cF;
      }
    }
    cx<R> Js[3], M[3];  // J_e + J_i and M of this triangle at the point
    for (int c = 0; c < 3; ++c) {
      Js[c] = rel[c] * se[0] - se[1 + c] + rel[c] * si[0] - si[1 + c];
      M[c] = rel[c] * sM[0] - sM[1 + c];
    }
    // n x (J_e + J_i), n x M and n x X
    cx<R> nJ[3], nM[3];
    nJ[0] = nrm[1] * Js[2] - nrm[2] * Js[1];
    nJ[1] = nrm[2] * Js[0] - nrm[0] * Js[2];
    nJ[2] = nrm[0] * Js[1] - nrm[1] * Js[0];
    nM[0] = nrm[1] * M[2] - nrm[2] * M[1];
    nM[1] = nrm[2] * M[0] - nrm[0] * M[2];
    nM[2] = nrm[0] * M[1] - nrm[1] * M[0];
    const R nX[3] = {nrm[1] * X[2] - nrm[2] * X[1], nrm[2] * X[0] - nrm[0] * X[2], nrm[0] * X[1] - nrm[1] * X[0]};
    const cx<R> XJ = dot3(X, Js), XnM = dot3(X, nM);
    const cx<R> hterm = dot3(X, WH) + divX * wH;
    v0 += w * (dot3(X, WE) + divX * wE);
    v1 += w * hterm;
    // Eq. 13: <X, dH> - <sigma n x X, E_e^+>, side limits (J_e+J_i) x n / 2 and sigma M / 2
    v2 += w * (hterm - R(0.5) * dot3(X, nJ) - sg * dot3(nX, E[0]) - (R(0.5) * sg) * dot3(X, M));
    // Eq. 14: <X, J_e + J_i> - <sigma X, E_i^->, side limit n x M / 2
    v3 += w * (XJ - sg * dot3(X, E[1]) - (R(0.5) * sg) * XnM);
  }
  cx<R>* o = val + gid * 4;
  o[0] = v0;
  o[1] = v1;
  o[2] = v2;
  o[3] = v3;
}

template <typename R>
__global__ void k_rows(const cx<R>* __restrict__ val, const int32_t* __restrict__ rowsrc, int64_t N,
                       cx<R>* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  y[i] = val[rowsrc[2 * i]] + val[rowsrc[2 * i + 1]];
}

template <typename R>
PrecData<R>& pdata(scabem_op* op);
template <>
PrecData<float>& pdata<float>(scabem_op* op) {
  return op->f;
}
template <>
PrecData<double>& pdata<double>(scabem_op* op) {
  return op->d;
}

}  // namespace

template <typename R>
int apply_one(scabem_op* op, const cx<R>* x, cx<R>* y, cudaStream_t s) {
  PrecData<R>& pd = pdata<R>(op);
  const int64_t nt = op->nt, Q = op->Q;
  const int n0 = op->n[0], n1 = op->n[1], n2 = op->n[2];
  const int64_t ng = (int64_t)n0 * n1 * n2;
  const int p3 = op->p * op->p * op->p;
  prof_mark(op, s);
  k_summ<R><<<(int)cdiv(nt, 128), 128, 0, s>>>(x, op->unk, op->cX, op->tri, nt, pd.summ);
  CK(cudaGetLastError());
  prof_mark(op, s);
  CK(cudaMemsetAsync(pd.src, 0, sizeof(cx<R>) * NFIELD_IN * ng, s));
  k_project<R><<<(int)cdiv(Q * p3, 256), 256, 0, s>>>(pd.summ, op->qp, op->qw, op->tri, op->base, pd.L, Q, op->q,
                                                       op->p, n0, n1, n2, pd.src);
  CK(cudaGetLastError());
  prof_mark(op, s);
  int rc = fft_conv<R>(op, pd, s);
  if (rc) return rc;
  prof_mark(op, s);
  k_interp<R><<<(int)cdiv(Q * 2, 128), 128, 0, s>>>(pd.grid, op->base, pd.L, pd.dL, Q, op->p, n0, n1, n2, pd.fpt);
  CK(cudaGetLastError());
  prof_mark(op, s);
  if (op->npairs > 0) {
    k_near<R><<<(int)cdiv(Q * 2, 128), 128, 0, s>>>(pd.near, op->noff, op->nsrc, pd.summ, Q, op->q, pd.fpt);
    CK(cudaGetLastError());
  }
  prof_mark(op, s);
  k_test<R><<<(int)cdiv(nt * 3, 128), 128, 0, s>>>(pd.fpt, pd.summ, op->tri, op->cX, op->qp, op->qw, pd.sig, nt,
                                                    op->q, (R)op->ke, (R)op->ki, (R)op->ze, (R)op->zi, pd.val);
  CK(cudaGetLastError());
  k_rows<R><<<(int)cdiv(op->N, 256), 256, 0, s>>>(pd.val, op->rowsrc, op->N, y);
  CK(cudaGetLastError());
  prof_mark(op, s);
  return SCABEM_OK;
}

// Current summaries only (used by the field evaluation at probe points).
template <typename R>
int compute_summ(scabem_op* op, const cx<R>* x, cx<R>* summ, cudaStream_t s) {
  k_summ<R><<<(int)cdiv(op->nt, 128), 128, 0, s>>>(x, op->unk, op->cX, op->tri, op->nt, summ);
  CK(cudaGetLastError());
  return SCABEM_OK;
}

template int compute_summ<double>(scabem_op*, const cx<double>*, cx<double>*, cudaStream_t);
template int apply_one<float>(scabem_op*, const cx<float>*, cx<float>*, cudaStream_t);
template int apply_one<double>(scabem_op*, const cx<double>*, cx<double>*, cudaStream_t);
