// The matvec y = A x of the grid-accelerated operator (one right-hand side).
//
//  K1 k_summ     RWG coefficients -> per-triangle current summaries
//                J(r) = a (r - c_t) - beta for the exterior J, interior J and
//                exterior M sets (current reduction, Eqs. 10-12)
//  K2 k_project  point sources at the quadrature points spread onto the grid
//                by the Lagrange stencils (12 fields)
//  K3-5          fft_conv (fft.cu): 12 -> 16 grid potentials (A, phi, F, psi
//                of each medium, Eqs. 15-16)
//  K6-8 k_points per target triangle: potentials, gradients and curls at its
//                quadrature points (interpolation), plus the near-field
//                precorrection (exact minus grid panel moments), then the
//                Galerkin testing of Eqs. 1-3 (weak form), Eq. 13 and Eq. 14
//                (sigma-weighted, with the side-limit terms)
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

// K2a: one thread per quadrature point: the weighted point sources
// qsrc[Qi*12 + set*4 + {x, y, z, div}] of the exterior J, interior J and
// exterior M sets (J(r) = a (r - c) - beta, div J = 2a, times the weight).
template <typename R>
__global__ void k_qsrc(const cx<R>* __restrict__ summ, const double* __restrict__ qp, const double* __restrict__ qw,
                       const double* __restrict__ tri, int64_t Q, int q, cx<R>* __restrict__ qsrc) {
  int64_t Qi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (Qi >= Q) return;
  const int64_t t = Qi / q;
  const double* g = tri + 16 * t;
  const R w = (R)qw[Qi];
  const R rel[3] = {(R)(qp[3 * Qi] - g[9]), (R)(qp[3 * Qi + 1] - g[10]), (R)(qp[3 * Qi + 2] - g[11])};
  cx<R>* o = qsrc + Qi * NFIELD_IN;
#pragma unroll
  for (int set = 0; set < 3; ++set) {
    const cx<R>* s = summ + (3 * t + set) * 4;
    const cx<R> a = s[0];
#pragma unroll
    for (int c = 0; c < 3; ++c) o[set * 4 + c] = w * (rel[c] * a - s[1 + c]);
    o[set * 4 + 3] = (R(2) * w) * a;
  }
}

// K2b: projection as a gather.  Sixteen lanes per grid point that some
// stencil covers share its entries (two in flight per lane), sum
// W_slot(point) * qsrc[point] over 16-byte loads, and reduce the 24 real
// sums by a reduce-scatter over shuffles (each round halves the values a
// lane keeps); lanes with an even index then write three of them.  Points no
// stencil covers stay zero from set-up.  The sum order is fixed, so the
// result does not depend on thread timing.
constexpr int GATHER_LANES = 16;

// a[0..23] += w * (re, im of the 12 fields of row src)
__device__ __forceinline__ void add_row(float* a, float w, const cx<float>* src) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float4 u = __ldg(s4 + i);
    a[4 * i + 0] = fmaf(w, u.x, a[4 * i + 0]);
    a[4 * i + 1] = fmaf(w, u.y, a[4 * i + 1]);
    a[4 * i + 2] = fmaf(w, u.z, a[4 * i + 2]);
    a[4 * i + 3] = fmaf(w, u.w, a[4 * i + 3]);
  }
}
__device__ __forceinline__ void add_row(double* a, double w, const cx<double>* src) {
  const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const double2 u = __ldg(s2 + i);
    a[2 * i + 0] = fma(w, u.x, a[2 * i + 0]);
    a[2 * i + 1] = fma(w, u.y, a[2 * i + 1]);
  }
}

// One reduce-scatter round over lanes l and l ^ M: the lane with bit M set
// keeps the upper half of its H values, the other the lower half.
template <int H, int M, typename R>
__device__ __forceinline__ void rs_round(const R* a, R* b, bool up) {
#pragma unroll
  for (int i = 0; i < H / 2; ++i) {
    const R send = up ? a[i] : a[i + H / 2];
    const R keep = up ? a[i + H / 2] : a[i];
    b[i] = keep + __shfl_xor_sync(0xffffffffu, send, M);
  }
}

template <typename R>
__global__ void k_gather(const cx<R>* __restrict__ qsrc, const int32_t* __restrict__ gpt,
                         const int32_t* __restrict__ goff, const int32_t* __restrict__ gq, const R* __restrict__ gw,
                         int64_t ngnz, int64_t ng, cx<R>* __restrict__ grids) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / GATHER_LANES;
  const int l = threadIdx.x & (GATHER_LANES - 1);
  R a[2 * NFIELD_IN];
#pragma unroll
  for (int f = 0; f < 2 * NFIELD_IN; ++f) a[f] = R(0);
  if (i < ngnz) {
    const int e1 = goff[i + 1];
    for (int e = goff[i] + l; e < e1; e += 2 * GATHER_LANES) {
      const int e2 = e + GATHER_LANES;
      const int qa = gq[e];
      const R wa = gw[e];
      const int qb = e2 < e1 ? gq[e2] : qa;
      const R wb = e2 < e1 ? gw[e2] : R(0);
      add_row(a, wa, qsrc + (int64_t)qa * NFIELD_IN);
      add_row(a, wb, qsrc + (int64_t)qb * NFIELD_IN);
    }
  }
  // every lane reaches the shuffles (no early exit above)
  R b[12], c[6], d[3];
  rs_round<24, 8>(a, b, l & 8);
  rs_round<12, 4>(b, c, l & 4);
  rs_round<6, 2>(c, d, l & 2);
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] += __shfl_xor_sync(0xffffffffu, d[k], 1);
  if (i < ngnz && (l & 1) == 0) {
    const int64_t g = gpt[i];
    const int v0 = ((l & 8) ? 12 : 0) + ((l & 4) ? 6 : 0) + ((l & 2) ? 3 : 0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int v = v0 + k;  // real sum v = field v / 2, part v % 2
      reinterpret_cast<R*>(grids + (v >> 1) * ng + g)[v & 1] = d[k];
    }
  }
}

template <typename R>
const R* gather_weights(scabem_op* op);
template <>
const float* gather_weights<float>(scabem_op* op) {
  return op->gwf;
}
template <>
const double* gather_weights<double>(scabem_op* op) {
  return op->gwd;
}

// Interpolated potentials of one medium at quadrature point Qi.  Record
// (NREC): A(3) phi grad phi(3) curl A(3) F(3) psi grad psi(3) curl F(3).
template <typename R>
__device__ __forceinline__ void interp_point(const cx<R>* __restrict__ grids, const int32_t* __restrict__ base,
                                             const R* __restrict__ L, const R* __restrict__ dL, int64_t Qi, int med,
                                             int p, int64_t ng, int n1, int n2, cx<R>* rec) {
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
  // two groups of 4 fields: (A, phi) of the J set, then (F, psi) of the M set
  for (int h = 0; h < 2; ++h) {
    cx<R> v[4], gx[4], gy[4], gz[4];
    for (int f = 0; f < 4; ++f) v[f] = gx[f] = gy[f] = gz[f] = czero<R>();
    const cx<R>* gm = grids + (int64_t)(med * 8 + 4 * h) * ng;
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j) {
        const R wxy = Lx[i] * Ly[j], dxy = dx[i] * Ly[j], xdy = Lx[i] * dy[j];
        const int64_t rowi = ((int64_t)(b0 + i) * n1 + (b1 + j)) * n2 + b2;
        for (int k = 0; k < p; ++k) {
          const R w = wxy * Lz[k], wx = dxy * Lz[k], wy = xdy * Lz[k], wz = wxy * dz[k];
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            const cx<R> gv = gm[f * ng + rowi + k];
            axpy(v[f], w, gv);
            axpy(gx[f], wx, gv);
            axpy(gy[f], wy, gv);
            axpy(gz[f], wz, gv);
          }
        }
      }
    cx<R>* r = rec + 10 * h;
    r[0] = v[0];
    r[1] = v[1];
    r[2] = v[2];
    r[3] = v[3];
    r[4] = gx[3];
    r[5] = gy[3];
    r[6] = gz[3];
    r[7] = gy[2] - gz[1];
    r[8] = gz[0] - gx[2];
    r[9] = gx[1] - gy[0];
  }
}

// One near record (dP0, dP1, dQ, dC) applied to the J and the M source of a
// pair: A += a dP1 - beta dP0, phi += 2a dP0, grad phi += 2a dQ,
// curl A += a dC - dQ x beta.
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

// Near-field precorrection of one (target point a of triangle t, medium).
template <typename R>
__device__ __forceinline__ void near_point(const cx<R>* __restrict__ corr, const int32_t* __restrict__ noff,
                                           const int32_t* __restrict__ nsrc, const cx<R>* __restrict__ summ,
                                           int64_t t, int a, int med, int q, cx<R>* rec) {
  const R sgnm = med == 1 ? R(-1) : R(1);  // interior M = -M
  cx<R>* accJ = rec;
  cx<R>* accM = rec + 10;
  const int j0 = noff[t], j1 = noff[t + 1];
  // records are [pair][component][point][medium]: the 2q threads of a
  // triangle read each component as one contiguous run
  const int cs = 2 * q;                     // component stride
  const int64_t stride = (int64_t)NCORR * cs;  // complex per pair
  const cx<R>* base = corr + (int64_t)a * 2 + med;
  int j = j0;
  for (; j + 1 < j1; j += 2) {
    cx<R> dA[NCORR], dB[NCORR];
    const int64_t sA = nsrc[j], sB = nsrc[j + 1];
    const cx<R>* pA = base + (int64_t)j * stride;
    const cx<R>* pB = pA + stride;
#pragma unroll
    for (int c = 0; c < NCORR; ++c) {
      dA[c] = pA[c * cs];
      dB[c] = pB[c * cs];
    }
    near_accumulate(dA, summ + (3 * sA + med) * 4, summ + (3 * sA + 2) * 4, sgnm, accJ, accM);
    near_accumulate(dB, summ + (3 * sB + med) * 4, summ + (3 * sB + 2) * 4, sgnm, accJ, accM);
  }
  if (j < j1) {
    cx<R> dA[NCORR];
    const int64_t sA = nsrc[j];
    const cx<R>* pA = base + (int64_t)j * stride;
#pragma unroll
    for (int c = 0; c < NCORR; ++c) dA[c] = pA[c * cs];
    near_accumulate(dA, summ + (3 * sA + med) * 4, summ + (3 * sA + 2) * 4, sgnm, accJ, accM);
  }
}

template <typename R>
__device__ __forceinline__ cx<R> dot3(const R* X, const cx<R>* V) {
  return X[0] * V[0] + X[1] * V[1] + X[2] * V[2];
}

// Tested values of local edge kk of triangle t from the records of its
// points (recs[(a*2 + medium)*NREC]): type 0 <X, E_e - E_i>, 1 <X, H_e - H_i>
// (weak forms), 2 Eq. 13, 3 Eq. 14.
template <typename R>
__device__ __forceinline__ void test_edge(const cx<R>* recs, const cx<R>* __restrict__ summ,
                                          const double* __restrict__ tri, const double* __restrict__ cX,
                                          const double* __restrict__ qp, const double* __restrict__ qw,
                                          const R* __restrict__ sig, int64_t t, int kk, int q, R ke, R ki, R ze,
                                          R zi, cx<R>* out) {
  const double* g = tri + 16 * t;
  const R cxk = (R)cX[3 * t + kk];
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
      const cx<R>* r = recs + (a * 2 + m) * NREC;
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
  out[0] = v0;
  out[1] = v1;
  out[2] = v2;
  out[3] = v3;
}

// K6-8: one CTA per PT_TRI target triangles.  Phase 1: thread (triangle,
// point, medium) interpolates its record and adds the near corrections, into
// shared memory.  Phase 2: thread (triangle, local edge) tests.
constexpr int PT_TRI = 16;

template <typename R>
__global__ void k_points(const cx<R>* __restrict__ grids, const int32_t* __restrict__ base, const R* __restrict__ L,
                         const R* __restrict__ dL, const cx<R>* __restrict__ corr, const int32_t* __restrict__ noff,
                         const int32_t* __restrict__ nsrc, const cx<R>* __restrict__ summ,
                         const double* __restrict__ tri, const double* __restrict__ cX, const double* __restrict__ qp,
                         const double* __restrict__ qw, const R* __restrict__ sig, int64_t nt, int q, int p, int n0,
                         int n1, int n2, R ke, R ki, R ze, R zi, int has_near, cx<R>* __restrict__ val) {
  extern __shared__ unsigned char smem_raw[];
  cx<R>* recs = reinterpret_cast<cx<R>*>(smem_raw);  // [PT_TRI][q][2][NREC]
  const int64_t t0 = (int64_t)blockIdx.x * PT_TRI;
  const int per = 2 * q;
  const int tl = threadIdx.x / per;
  const int rem = threadIdx.x - tl * per;
  const int a = rem >> 1, med = rem & 1;
  const int64_t t = t0 + tl;
  const int64_t ng = (int64_t)n0 * n1 * n2;
  if (tl < PT_TRI && t < nt) {
    cx<R> rec[NREC];
    interp_point(grids, base, L, dL, t * q + a, med, p, ng, n1, n2, rec);
    if (has_near) near_point(corr, noff, nsrc, summ, t, a, med, q, rec);
    cx<R>* o = recs + ((int64_t)tl * per + a * 2 + med) * NREC;
#pragma unroll
    for (int c = 0; c < NREC; ++c) o[c] = rec[c];
  }
  __syncthreads();
  const int tt = threadIdx.x / 3, kk = threadIdx.x - (threadIdx.x / 3) * 3;
  const int64_t t2 = t0 + tt;
  if (tt < PT_TRI && t2 < nt) {
    cx<R> o[4];
    test_edge(recs + (int64_t)tt * per * NREC, summ, tri, cX, qp, qw, sig, t2, kk, q, ke, ki, ze, zi, o);
    cx<R>* dst = val + (t2 * 3 + kk) * 4;
    for (int c = 0; c < 4; ++c) dst[c] = o[c];
  }
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
  prof_mark(op, s);
  k_summ<R><<<(int)cdiv(nt, 128), 128, 0, s>>>(x, op->unk, op->cX, op->tri, nt, pd.summ);
  CK(cudaGetLastError());
  prof_mark(op, s);
  k_qsrc<R><<<(int)cdiv(Q, 128), 128, 0, s>>>(pd.summ, op->qp, op->qw, op->tri, Q, op->q, pd.qsrc);
  CK(cudaGetLastError());
  if (op->ngnz > 0) {
    k_gather<R><<<(int)cdiv(op->ngnz * GATHER_LANES, 256), 256, 0, s>>>(pd.qsrc, op->gpt, op->goff, op->gent,
                                                                        gather_weights<R>(op), op->ngnz, ng, pd.src);
    CK(cudaGetLastError());
  }
  prof_mark(op, s);
  int rc = fft_conv<R>(op, pd, s);
  if (rc) return rc;
  prof_mark(op, s);
  {
    const int threads = PT_TRI * (2 * op->q > 3 ? 2 * op->q : 3);
    const size_t sm = (size_t)PT_TRI * 2 * op->q * NREC * sizeof(cx<R>);
    CK(cudaFuncSetAttribute(k_points<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_points<R><<<(int)cdiv(nt, PT_TRI), threads, sm, s>>>(
        pd.grid, op->base, pd.L, pd.dL, pd.near, op->noff, op->nsrc, pd.summ, op->tri, op->cX, op->qp, op->qw, pd.sig,
        nt, op->q, op->p, n0, n1, n2, (R)op->ke, (R)op->ki, (R)op->ze, (R)op->zi, op->npairs > 0 ? 1 : 0, pd.val);
    CK(cudaGetLastError());
  }
  prof_mark(op, s);
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
