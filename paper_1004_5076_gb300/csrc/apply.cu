// The matvec y = A x of the grid-accelerated operator (one right-hand side).
//
//  K1 k_sources  RWG coefficients -> per-triangle current summaries
//                J(r) = a (r - c_t) - beta for the exterior J, interior J and
//                exterior M sets (current reduction, Eqs. 10-12), and the
//                weighted point sources at the quadrature points
//  K2 k_gather   point sources spread onto the grid by the Lagrange stencils
//                (12 fields), as a gather over the covered grid points
//  K3-5          fft_conv (fft.cu): 12 -> 16 grid potentials (A, phi, F, psi
//                of each medium, Eqs. 15-16)
//  K6-8 k_points per target triangle: potentials, gradients and curls at its
//                quadrature points (interpolation), plus the near-field
//                precorrection (exact minus grid panel moments), then the
//                Galerkin testing of Eqs. 1-3 (weak form), Eq. 13 and Eq. 14
//                (sigma-weighted, with the side-limit terms)
//                and the per-edge sums of the two triangles' tested values
//                into the rows
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

// a += s * b on (re, im) as one packed FP32x2 FMA in complex64.
__device__ __forceinline__ void axpy2(cx<float>& a, float s, cx<float> b) {
  const float2 r = __ffma2_rn(make_float2(s, s), make_float2(b.re, b.im), make_float2(a.re, a.im));
  a = mk(r.x, r.y);
}
__device__ __forceinline__ void axpy2(cx<double>& a, double s, cx<double> b) { axpy(a, s, b); }

// K1+K2a: one thread per quadrature point (point a of triangle t): the
// current summaries of t (as k_summ; written by the thread of point 0) and
// the point's weighted sources qsrc[Qi*12 + set*4 + {x, y, z, div}] of the
// exterior J, interior J and exterior M sets (J(r) = a (r - c) - beta,
// div J = 2a, times the quadrature weight); it also zeroes the output y.
template <typename R>
__global__ void k_sources(const cx<R>* __restrict__ x, const int32_t* __restrict__ unk,
                          const double* __restrict__ cX, const double* __restrict__ tri,
                          const double* __restrict__ qp, const double* __restrict__ qw, int64_t Q, int q,
                          cx<R>* __restrict__ summ, cx<R>* __restrict__ qsrc, cx<R>* __restrict__ y, int64_t N,
                          int64_t ldx, int64_t ldy) {
  const int64_t Qi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (Qi >= Q) return;
  {  // right-hand side blockIdx.y of a batch: its columns and workspaces
    const int64_t c = blockIdx.y;
    x += c * ldx;
    y += c * ldy;
    summ += c * (Q / q) * 12;
    qsrc += c * Q * 12;
  }
  // y is summed into by k_points (two terms per row)
  for (int64_t r = Qi; r < N; r += Q) y[r] = czero<R>();
  const int64_t t = Qi / q;
  const int a = (int)(Qi - t * q);
  const double* g = tri + 16 * t;
  R rel[3][3];
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) rel[k][c] = (R)(g[3 * k + c] - g[9 + c]);
  R ck[3];
  for (int k = 0; k < 3; ++k) ck[k] = (R)cX[3 * t + k];
  const R w = (R)qw[Qi];
  const R rq[3] = {(R)(qp[3 * Qi] - g[9]), (R)(qp[3 * Qi + 1] - g[10]), (R)(qp[3 * Qi + 2] - g[11])};
  cx<R>* o = qsrc + Qi * NFIELD_IN;
#pragma unroll
  for (int set = 0; set < 3; ++set) {
    cx<R> al = czero<R>(), b0 = al, b1 = al, b2 = al;
    for (int k = 0; k < 3; ++k) {
      const cx<R> j = ck[k] * coef_of(x, unk[(3 * t + k) * 3 + set]);
      al += j;
      b0 += rel[k][0] * j;
      b1 += rel[k][1] * j;
      b2 += rel[k][2] * j;
    }
    if (a == 0) {
      cx<R>* so = summ + (3 * t + set) * 4;
      so[0] = al;
      so[1] = b0;
      so[2] = b1;
      so[3] = b2;
    }
    o[set * 4 + 0] = w * (rq[0] * al - b0);
    o[set * 4 + 1] = w * (rq[1] * al - b1);
    o[set * 4 + 2] = w * (rq[2] * al - b2);
    o[set * 4 + 3] = (R(2) * w) * al;
  }
}

// K2b: projection as a gather.  One warp per grid point that some stencil
// covers: lane = portion * SL + slot reads 16-byte portion `portion` of the
// rows qsrc[point] of entries slot, slot + SL, ... (SL rows per load
// instruction, GATHER_INFLIGHT in flight), weighted by W_slot(point); the SL slot sums
// of a portion are then added by shuffles and the slot-0 lanes write their
// portion.  Points no stencil covers stay zero from set-up.  The sum order
// is fixed, so the result does not depend on thread timing.
constexpr int GATHER_INFLIGHT = 4;

template <typename R>
__device__ __forceinline__ void load_portion(const cx<R>* p, cx<R>* v);
template <>
__device__ __forceinline__ void load_portion<float>(const cx<float>* p, cx<float>* v) {
  const float4 u = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = mk(u.x, u.y);
  v[1] = mk(u.z, u.w);
}
template <>
__device__ __forceinline__ void load_portion<double>(const cx<double>* p, cx<double>* v) {
  v[0] = p[0];
}

template <typename R>
__global__ void k_gather(const cx<R>* __restrict__ qsrc, const int32_t* __restrict__ gpt,
                         const int32_t* __restrict__ goff, const int32_t* __restrict__ gq, const R* __restrict__ gw,
                         int64_t ngnz, int64_t ng, cx<R>* __restrict__ grids, int64_t cs_q, int64_t cs_g) {
  constexpr int CPP = 16 / (int)sizeof(cx<R>);  // complex per 16-byte portion
  qsrc += blockIdx.y * cs_q;  // right-hand side blockIdx.y of a batch
  grids += blockIdx.y * cs_g;
  constexpr int NPOR = NFIELD_IN / CPP;          // portions per row: 6 or 12
  constexpr int SL = 24 / NPOR;                  // rows per load instruction: 4 or 2
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int por = lane / SL, slot = lane - por * SL;
  const bool act = lane < NPOR * SL && i < ngnz;
  cx<R> acc[CPP];
#pragma unroll
  for (int c = 0; c < CPP; ++c) acc[c] = czero<R>();
  if (act) {
    const int e1 = goff[i + 1];
    for (int e = goff[i] + slot; e < e1; e += GATHER_INFLIGHT * SL) {
      int qe[GATHER_INFLIGHT];
      R we[GATHER_INFLIGHT];
#pragma unroll
      for (int u = 0; u < GATHER_INFLIGHT; ++u) {
        const int eu = e + u * SL;
        qe[u] = eu < e1 ? gq[eu] : gq[e];
        we[u] = eu < e1 ? gw[eu] : R(0);
      }
      cx<R> v[GATHER_INFLIGHT][CPP];
#pragma unroll
      for (int u = 0; u < GATHER_INFLIGHT; ++u) load_portion<R>(qsrc + (int64_t)qe[u] * NFIELD_IN + por * CPP, v[u]);
#pragma unroll
      for (int u = 0; u < GATHER_INFLIGHT; ++u)
#pragma unroll
        for (int c = 0; c < CPP; ++c) axpy2(acc[c], we[u], v[u][c]);
    }
  }
  // every lane reaches the shuffles (no early exit above)
#pragma unroll
  for (int o = 1; o < SL; o <<= 1)
#pragma unroll
    for (int c = 0; c < CPP; ++c) {
      acc[c].re += __shfl_xor_sync(0xffffffffu, acc[c].re, o);
      acc[c].im += __shfl_xor_sync(0xffffffffu, acc[c].im, o);
    }
  if (act && slot == 0) {
    const int64_t g = gpt[i];
#pragma unroll
    for (int c = 0; c < CPP; ++c) grids[(int64_t)(por * CPP + c) * ng + g] = acc[c];
  }
}

template <typename R>
const R* gather_dweights(scabem_op* op);
template <>
const float* gather_dweights<float>(scabem_op* op) {
  return op->gdf;
}
template <>
const double* gather_dweights<double>(scabem_op* op) {
  return op->gdd;
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

// The four potentials of one (grid point, medium, group) (32 contiguous bytes
// in complex64).
__device__ __forceinline__ void load_group(const cx<float>* p, cx<float>* v) {
  const float4 u0 = __ldg(reinterpret_cast<const float4*>(p));
  const float4 u1 = __ldg(reinterpret_cast<const float4*>(p) + 1);
  v[0] = mk(u0.x, u0.y);
  v[1] = mk(u0.z, u0.w);
  v[2] = mk(u1.x, u1.y);
  v[3] = mk(u1.z, u1.w);
}
__device__ __forceinline__ void load_group(const cx<double>* p, cx<double>* v) {
#pragma unroll
  for (int f = 0; f < 4; ++f) v[f] = p[f];
}

// Two consecutive complex values of shared memory on a 16-byte boundary.
__device__ __forceinline__ void load_pair_smem(const cx<float>* p, cx<float>* v) {
  const float4 u = *reinterpret_cast<const float4*>(p);
  v[0] = mk(u.x, u.y);
  v[1] = mk(u.z, u.w);
}
__device__ __forceinline__ void load_pair_smem(const cx<double>* p, cx<double>* v) {
  v[0] = p[0];
  v[1] = p[1];
}

// Two consecutive complex values starting on a 16-byte boundary.
__device__ __forceinline__ void load_pair(const cx<float>* p, cx<float>* v) {
  const float4 u = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = mk(u.x, u.y);
  v[1] = mk(u.z, u.w);
}
__device__ __forceinline__ void load_pair(const cx<double>* p, cx<double>* v) {
  v[0] = p[0];
  v[1] = p[1];
}

// Interpolated potentials of one medium at quadrature point Qi, group h of
// the record (NREC = 2 x 10): h = 0 A(3) phi grad phi(3) curl A(3) from the
// J fields, h = 1 F(3) psi grad psi(3) curl F(3) from the M fields.  The
// grid is point-major: point g holds its 16 potentials at grids[16 g ..].
template <typename R, int p>
__device__ __forceinline__ void interp_group(const cx<R>* __restrict__ grids, const int32_t* __restrict__ base,
                                             const R* __restrict__ L, const R* __restrict__ dL, int64_t Qi, int med,
                                             int h, int n1, int n2, cx<R>* r) {
  R Lx[p], Ly[p], Lz[p], dx[p], dy[p], dz[p];
#pragma unroll
  for (int i = 0; i < p; ++i) {
    Lx[i] = L[(3 * Qi + 0) * p + i];
    Ly[i] = L[(3 * Qi + 1) * p + i];
    Lz[i] = L[(3 * Qi + 2) * p + i];
    dx[i] = dL[(3 * Qi + 0) * p + i];
    dy[i] = dL[(3 * Qi + 1) * p + i];
    dz[i] = dL[(3 * Qi + 2) * p + i];
  }
  const int b0 = base[3 * Qi], b1 = base[3 * Qi + 1], b2 = base[3 * Qi + 2];
  cx<R> v[4], gx[4], gy[4], gz[4];
  for (int f = 0; f < 4; ++f) v[f] = gx[f] = gy[f] = gz[f] = czero<R>();
  const cx<R>* gm = grids + 4 * (med * 2 + h);
#pragma unroll
  for (int i = 0; i < p; ++i)
#pragma unroll
    for (int j = 0; j < p; ++j) {
      const R wxy = Lx[i] * Ly[j], dxy = dx[i] * Ly[j], xdy = Lx[i] * dy[j];
      const int64_t rowi = ((int64_t)(b0 + i) * n1 + (b1 + j)) * n2 + b2;
#pragma unroll
      for (int k = 0; k < p; ++k) {
        const R w = wxy * Lz[k], wx = dxy * Lz[k], wy = xdy * Lz[k], wz = wxy * dz[k];
        cx<R> gv[4];
        load_group(gm + (rowi + k) * NFIELD_OUT, gv);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          axpy2(v[f], w, gv[f]);
          axpy2(gx[f], wx, gv[f]);
          axpy2(gy[f], wy, gv[f]);
          axpy2(gz[f], wz, gv[f]);
        }
      }
    }
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

// The same sums in complex64 with the accumulator split as acc = P + j Q:
// x s adds (s.re, s.re) * (x.re, x.im) to P and (s.im, s.im) * (x.re, x.im)
// to Q, so that every record value enters the packed FMAs as the (re, im)
// pair it is loaded as, and only the few source factors are duplicated.
__device__ __forceinline__ void near_pq(const cx<float>* d, const cx<float>* sv, float2* P, float2* Q) {
  float2 x[NCORR];
#pragma unroll
  for (int c = 0; c < NCORR; ++c) x[c] = make_float2(d[c].re, d[c].im);
  const float2 ar = make_float2(sv[0].re, sv[0].re), ai = make_float2(sv[0].im, sv[0].im);
  const float2 a2r = make_float2(2.f * sv[0].re, 2.f * sv[0].re), a2i = make_float2(2.f * sv[0].im, 2.f * sv[0].im);
  float2 br[3], bi[3], nbr[3], nbi[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    br[c] = make_float2(sv[1 + c].re, sv[1 + c].re);
    bi[c] = make_float2(sv[1 + c].im, sv[1 + c].im);
    nbr[c] = make_float2(-sv[1 + c].re, -sv[1 + c].re);
    nbi[c] = make_float2(-sv[1 + c].im, -sv[1 + c].im);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    P[c] = __ffma2_rn(x[1 + c], ar, P[c]);  // A += a dP1 - beta dP0
    Q[c] = __ffma2_rn(x[1 + c], ai, Q[c]);
    P[c] = __ffma2_rn(x[0], nbr[c], P[c]);
    Q[c] = __ffma2_rn(x[0], nbi[c], Q[c]);
    P[4 + c] = __ffma2_rn(x[4 + c], a2r, P[4 + c]);  // grad phi += 2a dQ
    Q[4 + c] = __ffma2_rn(x[4 + c], a2i, Q[4 + c]);
    P[7 + c] = __ffma2_rn(x[7 + c], ar, P[7 + c]);  // curl A += a dC
    Q[7 + c] = __ffma2_rn(x[7 + c], ai, Q[7 + c]);
  }
  P[3] = __ffma2_rn(x[0], a2r, P[3]);  // phi += 2a dP0
  Q[3] = __ffma2_rn(x[0], a2i, Q[3]);
  // curl A -= dQ x beta
  P[7] = __ffma2_rn(x[5], nbr[2], P[7]);
  Q[7] = __ffma2_rn(x[5], nbi[2], Q[7]);
  P[7] = __ffma2_rn(x[6], br[1], P[7]);
  Q[7] = __ffma2_rn(x[6], bi[1], Q[7]);
  P[8] = __ffma2_rn(x[6], nbr[0], P[8]);
  Q[8] = __ffma2_rn(x[6], nbi[0], Q[8]);
  P[8] = __ffma2_rn(x[4], br[2], P[8]);
  Q[8] = __ffma2_rn(x[4], bi[2], Q[8]);
  P[9] = __ffma2_rn(x[4], nbr[1], P[9]);
  Q[9] = __ffma2_rn(x[4], nbi[1], Q[9]);
  P[9] = __ffma2_rn(x[5], br[0], P[9]);
  Q[9] = __ffma2_rn(x[5], bi[0], Q[9]);
}

// Near-field accumulation state of one lane: complex64 keeps acc = P + j Q
// through the near loop (near_pq); complex128 keeps acc itself (near_part).
template <typename R>
struct NearAcc;
template <>
struct NearAcc<float> {
  float2 P[NREC / 2], Q[NREC / 2];
  __device__ __forceinline__ void begin(const cx<float>* acc) {
#pragma unroll
    for (int c = 0; c < NREC / 2; ++c) {
      P[c] = make_float2(acc[c].re, acc[c].im);
      Q[c] = make_float2(0.f, 0.f);
    }
  }
  __device__ __forceinline__ void add(const cx<float>* d, const cx<float>* sv) { near_pq(d, sv, P, Q); }
  __device__ __forceinline__ void end(cx<float>* acc) const {
#pragma unroll
    for (int c = 0; c < NREC / 2; ++c) acc[c] = mk(P[c].x - Q[c].y, P[c].y + Q[c].x);
  }
};

// One near record (dP0, dP1, dQ, dC) applied to source summary sv (a, beta):
// A += a dP1 - beta dP0, phi += 2a dP0, grad phi += 2a dQ,
// curl A += a dC - dQ x beta (the same for F, psi of an M source).
template <typename R>
__device__ __forceinline__ void near_part(const cx<R>* d, const cx<R>* sv, cx<R>* acc) {
  const cx<R> d0 = d[0];
  const cx<R> al = sv[0], al2 = R(2) * al;
  const cx<R> be[3] = {sv[1], sv[2], sv[3]};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cfma(acc[c], al, d[1 + c]);
    acc[c] -= be[c] * d0;
    cfma(acc[4 + c], al2, d[4 + c]);
    cfma(acc[7 + c], al, d[7 + c]);
  }
  cfma(acc[3], al2, d0);
  acc[7] -= d[5] * be[2] - d[6] * be[1];
  acc[8] -= d[6] * be[0] - d[4] * be[2];
  acc[9] -= d[4] * be[1] - d[5] * be[0];
}

template <>
struct NearAcc<double> {
  cx<double> a[NREC / 2];
  __device__ __forceinline__ void begin(const cx<double>* acc) {
#pragma unroll
    for (int c = 0; c < NREC / 2; ++c) a[c] = acc[c];
  }
  __device__ __forceinline__ void add(const cx<double>* d, const cx<double>* sv) { near_part(d, sv, a); }
  __device__ __forceinline__ void end(cx<double>* acc) const {
#pragma unroll
    for (int c = 0; c < NREC / 2; ++c) acc[c] = a[c];
  }
};

template <typename R>
__device__ __forceinline__ cx<R> dot3(const R* X, const cx<R>* V) {
  return X[0] * V[0] + X[1] * V[1] + X[2] * V[2];
}

// Weighted contributions of quadrature point a to the tested values of local
// edge kk of triangle t, from the point's records (recs[medium*NREC]):
// type 0 <X, E_e - E_i>, 1 <X, H_e - H_i> (weak forms), 2 Eq. 13, 3 Eq. 14.
template <typename R>
__device__ __forceinline__ void test_point(const cx<R>* recs, const cx<R>* __restrict__ summ,
                                           const double* __restrict__ tri, const R* __restrict__ tp,
                                           const R* __restrict__ sig, int64_t t, int kk, int a, int q, R ke, R ki,
                                           R ze, R zi, cx<R>* out) {
  const double* g = tri + 16 * t;
  const R nrm[3] = {(R)g[12], (R)g[13], (R)g[14]};
  const cx<R>* se = summ + (3 * t + 0) * 4;
  const cx<R>* si = summ + (3 * t + 1) * 4;
  const cx<R>* sM = summ + (3 * t + 2) * 4;
  const R kl[2] = {ke, ki}, zl[2] = {ze, zi};
  const int64_t Qa = t * q + a;
  const R* tq = tp + 16 * Qa;
  const R w = tq[3];
  const R sg = sig[Qa];
  const R divX = tq[13 + kk];
  R X[3], rel[3];
  for (int c = 0; c < 3; ++c) {
    X[c] = tq[4 + 3 * kk + c];
    rel[c] = tq[c];
  }
  cx<R> WE[3], WH[3], E[2][3];
  cx<R> wE = czero<R>(), wH = czero<R>();
  for (int c = 0; c < 3; ++c) WE[c] = WH[c] = czero<R>();
  for (int m = 0; m < 2; ++m) {
    const cx<R>* r = recs + m * NREC;
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
  out[0] = w * (dot3(X, WE) + divX * wE);
  out[1] = w * hterm;
  // Eq. 13: <X, dH> - <sigma n x X, E_e^+>, side limits (J_e+J_i) x n / 2 and sigma M / 2
  out[2] = w * (hterm - R(0.5) * dot3(X, nJ) - sg * dot3(nX, E[0]) - (R(0.5) * sg) * dot3(X, M));
  // Eq. 14: <X, J_e + J_i> - <sigma X, E_i^->, side limit n x M / 2
  out[3] = w * (XJ - sg * dot3(X, E[1]) - (R(0.5) * sg) * XnM);
}

// d out / d sg of the Eq. 13 and Eq. 14 tested values of local edge kk at
// point a (sg the normalised conductivity): d2 = w (-(n x X) . E_e - X . M / 2),
// d3 = w (-X . E_i - X . (n x M) / 2), from the point's records.
template <typename R>
__device__ __forceinline__ void test_point_sigma(const cx<R>* recs, const cx<R>* __restrict__ summ,
                                                 const double* __restrict__ tri, const R* __restrict__ tp, int64_t t,
                                                 int kk, int a, int q, R ke, R ki, R ze, R zi, cx<R>& d2,
                                                 cx<R>& d3) {
  const double* g = tri + 16 * t;
  const R nrm[3] = {(R)g[12], (R)g[13], (R)g[14]};
  const cx<R>* sM = summ + (3 * t + 2) * 4;
  const R* tq = tp + 16 * (t * q + a);
  const R w = tq[3];
  R X[3], rel[3];
  for (int c = 0; c < 3; ++c) {
    X[c] = tq[4 + 3 * kk + c];
    rel[c] = tq[c];
  }
  const R kl[2] = {ke, ki}, zl[2] = {ze, zi};
  cx<R> E[2][3];
  for (int m = 0; m < 2; ++m) {
    const cx<R>* r = recs + m * NREC;
    const R k = kl[m], z = zl[m];
    for (int c = 0; c < 3; ++c)
      E[m][c] = -z * (k * mulj(r[c]) + (R(1) / k) * mulj(r[4 + c])) - r[17 + c];
  }
  cx<R> M[3], nM[3];
  for (int c = 0; c < 3; ++c) M[c] = rel[c] * sM[0] - sM[1 + c];
  nM[0] = nrm[1] * M[2] - nrm[2] * M[1];
  nM[1] = nrm[2] * M[0] - nrm[0] * M[2];
  nM[2] = nrm[0] * M[1] - nrm[1] * M[0];
  const R nX[3] = {nrm[1] * X[2] - nrm[2] * X[1], nrm[2] * X[0] - nrm[0] * X[2], nrm[0] * X[1] - nrm[1] * X[0]};
  d2 = -w * (dot3(nX, E[0]) + R(0.5) * dot3(X, M));
  d3 = -w * (dot3(X, E[1]) + R(0.5) * dot3(X, nM));
}

// Bulk asynchronous global -> shared copies (the TMA unit, cp.async.bulk)
// completing on an mbarrier, and bounded waits on it.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// The near records are read once per apply: their copies carry an L2
// evict-first policy, so that the stream of records does not push the
// apply's reused data (grids, sources, geometry) and the caller's vectors out
// of L2.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
// The arrival of one thread that expects `bytes` of copies on `bar`, and one
// bulk copy completing its bytes there (several copies may share one arrival).
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// one arrival that also expects `bytes` of transaction, then the copy
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  mbar_expect_tx(bar, bytes);
  bulk_copy(dst, src, bytes, bar);
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// Wait for the phase of the given parity; false after about a second.
constexpr uint64_t WAIT_LIMIT_NS = 1000000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (gtimer_ns() - t0 > WAIT_LIMIT_NS) return false;
  }
}

// Self-test of the bounded waits: one warp waits on an mbarrier that no
// arrival or copy ever completes, through the same mbar_wait as the record
// rings; when the wait gives up it reports through *tmo exactly as they do.
__global__ void k_wait_selftest(int* __restrict__ tmo) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncwarp();
  const bool ok = __all_sync(0xffffffffu, mbar_wait(&bar, 0));
  if (!ok && threadIdx.x == 0) atomicOr(tmo, 1);
}

// K6-8: one warp per target triangle t, PT_WARPS triangles per CTA; warps
// never wait on one another.
//  Phase 1: lane (point a, medium, record group h), 4q lanes, interpolates
//    its 10 record values, then adds the near corrections.  The triangle's
//    near records are one contiguous run (pairs noff[t] .. noff[t+1]); they
//    stream through a per-warp ring of PT_NSTG stages of PT_KP pairs, one
//    bulk copy per stage issued by lane 0, the next stages in flight while
//    one is consumed (the first ones during the interpolation).  A stage
//    that does not arrive within the wait limit sets *tmo and ends the
//    triangle's near loop after its copies in flight have landed.
//  Phase 2: lane (local edge kk, point a), 3q lanes, forms the point's
//    weighted tested values; phase 3: lane (kk, value type) sums them over the
//    points in point order.
constexpr int PT_WARPS = 4;
constexpr int PT_NSTG = 2;  // 2 stages of 4 pairs: the bytes in flight of 4 stages of 2, with half the
constexpr int PT_KP = 4;    // stages' waits, fences and copy issues per pair

// complex values of per-warp shared memory: the ring, which the records and
// point parts of phases 2-3 reuse once the near loop is done
__host__ __device__ constexpr int pt_warp_complex(int q) {
  return PT_NSTG * PT_KP * NCORR * 2 * q > 2 * q * NREC + 3 * q * 4 ? PT_NSTG * PT_KP * NCORR * 2 * q
                                                                     : 2 * q * NREC + 3 * q * 4;
}
// bytes of shared memory per CTA: rings, then one mbarrier per stage and warp
__host__ __device__ constexpr size_t pt_smem_bytes(int q, size_t csize) {
  return (size_t)PT_WARPS * pt_warp_complex(q) * csize + (size_t)PT_WARPS * PT_NSTG * sizeof(uint64_t);
}

// SENS = true (conductivity sensitivity): instead of testing into y, the
// kernel writes hs[t q + a] = eta0 sum_kk (lam_row2 d2 + lam_row3 d3), the
// derivative of lam^T A x with respect to the conductivity [S] at the point.
//
// QT > 0 fixes q at compile time (then every shared-memory offset of a record
// is an immediate); QT = 0 takes the argument.  Lanes past the 4q of phase 1
// repeat lane 4q - 4 .. 4q - 1's work without storing it, so that the near
// loop runs without divergence.
template <typename R, int P, bool SENS = false, int QT = 0>
__global__ void __launch_bounds__(PT_WARPS * 32, sizeof(R) == 4 ? (P == 4 ? 4 : 6) : 3) k_points(
    const cx<R>* __restrict__ grids, const int32_t* __restrict__ base, const R* __restrict__ L,
    const R* __restrict__ dL, const cx<R>* __restrict__ corr, const int32_t* __restrict__ noff,
    const int32_t* __restrict__ nsrc, const cx<R>* __restrict__ summ, const double* __restrict__ tri,
    const R* __restrict__ tp, const R* __restrict__ sig, int64_t nt, int q_arg, int n0, int n1, int n2, R ke, R ki,
    R ze, R zi, int has_near, const int32_t* __restrict__ valrow, cx<R>* __restrict__ y, int* __restrict__ tmo,
    const cx<R>* __restrict__ lam, cx<R>* __restrict__ hs) {
  const int q = QT > 0 ? QT : q_arg;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * PT_WARPS + warp;
  if (t >= nt) return;  // whole warp; no CTA-wide barrier below
  const int pairc = NCORR * 2 * q;  // complex per pair: [point][medium][component]
  cx<R>* ring = reinterpret_cast<cx<R>*>(smem_raw) + (int64_t)warp * pt_warp_complex(q);
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<cx<R>*>(smem_raw) + PT_WARPS * pt_warp_complex(q)) +
                   warp * PT_NSTG;
  cx<R>* recs = ring;                 // [q][2][NREC], after the near loop
  cx<R>* part = recs + 2 * q * NREC;  // [3][q][4]

  const bool act = lane < 4 * q;
  const int a = min(lane >> 2, q - 1), med = (lane >> 1) & 1, h = lane & 1;
  const int j0 = has_near ? noff[t] : 0, j1 = has_near ? noff[t + 1] : 0;
  const int nst = (j1 - j0 + PT_KP - 1) / PT_KP;
  const unsigned pair_bytes = (unsigned)(pairc * sizeof(cx<R>));
  // stage st -> slot st % PT_NSTG, issued by lane 0
  auto issue = [&](int st) {
    const int pj = j0 + st * PT_KP;
    const int np = min(PT_KP, j1 - pj);
    fence_proxy_async();  // earlier reads of the slot come before the copy
    bulk_load(ring + (st % PT_NSTG) * PT_KP * pairc, corr + (int64_t)pj * pairc, np * pair_bytes,
              bars + st % PT_NSTG);
  };
  if (nst > 0) {
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < PT_NSTG; ++i) mbar_init(bars + i, 1);
      mbar_init_fence();
      for (int st = 0; st < PT_NSTG - 1 && st < nst; ++st) issue(st);
    }
    __syncwarp();
  }
  // source triangles of the pairs, 32 at a time in the lanes (one block ahead)
  const int npair = j1 - j0;
  int src_nxt = lane < npair ? nsrc[j0 + lane] : 0, src_cur = 0;
  cx<R> acc[NREC / 2];
  interp_group<R, P>(grids, base, L, dL, t * q + a, med, h, n1, n2, acc);
  if (nst > 0) {
    const int set = h ? 2 : med;  // source J of this medium, or M
    // the interior medium sees -M: accumulate -acc + sum, then negate back
    const bool neg = h && med;
    if (neg)
#pragma unroll
      for (int c = 0; c < NREC / 2; ++c) acc[c] = -acc[c];
    NearAcc<R> na;
    na.begin(acc);
    int st = 0;
    bool ok = true;
    for (; st < nst; ++st) {
      if (lane == 0 && st + PT_NSTG - 1 < nst) issue(st + PT_NSTG - 1);  // slot consumed at st - 1
      ok = __all_sync(0xffffffffu, mbar_wait(bars + st % PT_NSTG, (st / PT_NSTG) & 1));
      if (!ok) break;
      const cx<R>* rs = ring + (st % PT_NSTG) * PT_KP * pairc + (a * 2 + med) * NCORR;
#pragma unroll
      for (int k = 0; k < PT_KP; ++k) {
        const int jj = st * PT_KP + k;  // pair within the triangle (warp-uniform)
        if (jj < npair) {
          if ((jj & 31) == 0) {
            src_cur = src_nxt;
            src_nxt = jj + 32 + lane < npair ? nsrc[j0 + jj + 32 + lane] : 0;
          }
          const int64_t sj = __shfl_sync(0xffffffffu, src_cur, jj & 31);
          cx<R> d[NCORR], sv[4];
          load_group(summ + (3 * sj + set) * 4, sv);
#pragma unroll
          for (int c = 0; c < NCORR; c += 2) load_pair_smem(rs + k * pairc + c, d + c);
          na.add(d, sv);
        }
      }
      __syncwarp();
    }
    if (!ok) {
      // stages st .. min(st + PT_NSTG - 1, nst - 1) were issued: let them land
      for (int s2 = st; s2 < nst && s2 < st + PT_NSTG; ++s2) (void)mbar_wait(bars + s2 % PT_NSTG, (s2 / PT_NSTG) & 1);
      if (lane == 0) atomicOr(tmo, 1);
    }
    __syncwarp();  // every lane is done with the ring before it holds records
    na.end(acc);
    if (neg)
#pragma unroll
      for (int c = 0; c < NREC / 2; ++c) acc[c] = -acc[c];
  }
  if (act) {
    cx<R>* o = recs + (a * 2 + med) * NREC + 10 * h;
#pragma unroll
    for (int c = 0; c < NREC / 2; ++c) o[c] = acc[c];
  }
  __syncwarp();
  if constexpr (SENS) {
    if (lane < 3 * q) {
      const int kk = lane / q, pa = lane - kk * q;
      cx<R> d2, d3;
      test_point_sigma(recs + pa * 2 * NREC, summ, tri, tp, t, kk, pa, q, ke, ki, ze, zi, d2, d3);
      const int r2 = valrow[(t * 3 + kk) * 4 + 2], r3 = valrow[(t * 3 + kk) * 4 + 3];
      cx<R> c = czero<R>();
      if (r2 >= 0) c += lam[r2] * d2;
      if (r3 >= 0) c += lam[r3] * d3;
      part[kk * q + pa] = c;
    }
    __syncwarp();
    if (lane < q) hs[t * q + lane] = R(ETA0) * (part[lane] + part[q + lane] + part[2 * q + lane]);
    return;
  }
  if (lane < 3 * q) {
    const int kk = lane / q, pa = lane - kk * q;
    cx<R> o[4];
    test_point(recs + pa * 2 * NREC, summ, tri, tp, sig, t, kk, pa, q, ke, ki, ze, zi, o);
    cx<R>* d = part + (kk * q + pa) * 4;
#pragma unroll
    for (int c = 0; c < 4; ++c) d[c] = o[c];
  }
  __syncwarp();
  if (lane < 12) {
    const int kk = lane >> 2, c = lane & 3;
    const cx<R>* sp = part + kk * q * 4 + c;
    cx<R> v = czero<R>();
    for (int pa = 0; pa < q; ++pa) v += sp[pa * 4];
    // each row is the sum of exactly two such values (the edge's two
    // triangles) added to a zeroed word, so the result does not depend on
    // which arrives first
    const int row = valrow[(t * 3 + kk) * 4 + c];
    if (row >= 0) {
      atomicAdd(&y[row].re, v.re);
      atomicAdd(&y[row].im, v.im);
    }
  }
}


// K6-8 for a batch of ncol right-hand sides: one CTA per target triangle
// t = blockIdx.x.  Thread T works on column T / 4q as lane (point, medium,
// group) T mod 4q of k_points would, so the 4q lanes of each column are
// packed back to back (8 columns x 24 lanes = 6 full warps for q = 6, where
// a warp per column would leave 8 lanes of every warp idle).  The near
// records of t stream once through one ring shared by all threads (PB_NSTG
// stages of PB_KP pairs, filled by thread 0 with bulk copies), so each record
// leaves HBM once for all columns.  After consuming a stage every thread
// joins a CTA barrier that also combines the bounded waits' results: the
// slot is then free for the next copy, and all threads leave the stage loop
// together when a wait expired.  Testing (3q tasks per column) and the row
// sums (12 per column) are packed the same way, on a per-column area beside
// the ring.
constexpr int PB_NSTG = 2;  // 2 stages of 8 pairs: half the CTA barriers and waits of 4 stages of 4
constexpr int PB_KP = 8;

__host__ __device__ constexpr int pb_ring_complex(int q) { return PB_NSTG * PB_KP * NCORR * 2 * q; }
__host__ __device__ constexpr int pb_col_complex(int q) { return 2 * q * NREC + 3 * q * 4; }
__host__ __device__ constexpr size_t pb_smem_bytes(int q, int kc, size_t csize) {
  return ((size_t)pb_ring_complex(q) + (size_t)kc * pb_col_complex(q)) * csize + PB_NSTG * sizeof(uint64_t);
}
__host__ __device__ constexpr int pb_threads(int q, int ncol) { return (4 * q * ncol + 31) / 32 * 32; }

template <typename R, int P, int QT = 0>
__global__ void __launch_bounds__(KBATCH * 32, sizeof(R) == 4 ? (P == 4 ? 2 : 3) : 1) k_points_batch(
    const cx<R>* __restrict__ grids, const int32_t* __restrict__ base, const R* __restrict__ L,
    const R* __restrict__ dL, const cx<R>* __restrict__ corr, const int32_t* __restrict__ noff,
    const int32_t* __restrict__ nsrc, const cx<R>* __restrict__ summ, const double* __restrict__ tri,
    const R* __restrict__ tp, const R* __restrict__ sig, int64_t nt, int q_arg, int n0, int n1, int n2, R ke, R ki,
    R ze, R zi, int has_near, const int32_t* __restrict__ valrow, cx<R>* __restrict__ y, int* __restrict__ tmo,
    int64_t cs_grid, int64_t cs_summ, int64_t ldy, int ncol) {
  const int q = QT > 0 ? QT : q_arg;  // as in k_points
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int T = threadIdx.x, lane = T & 31;
  const int nl = 4 * q;                    // phase-1 tasks per column
  const bool act = T < ncol * nl;          // threads past them repeat a task of the last column, unstored
  const int col = act ? T / nl : ncol - 1;
  const int task = act ? T - col * nl : nl - 1;
  const int64_t t = blockIdx.x;
  const int pairc = NCORR * 2 * q;
  cx<R>* ring = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* area = ring + pb_ring_complex(q);  // per column: recs [q][2][NREC], then part [3][q][4]
  uint64_t* bars = reinterpret_cast<uint64_t*>(area + (int64_t)ncol * pb_col_complex(q));

  const int a = task >> 2, med = (task >> 1) & 1, h = task & 1;
  const int j0 = has_near ? noff[t] : 0, j1 = has_near ? noff[t + 1] : 0;
  const int nst = (j1 - j0 + PB_KP - 1) / PB_KP;  // the same for every thread of the CTA
  const unsigned pair_bytes = (unsigned)(pairc * sizeof(cx<R>));
  auto issue = [&](int st) {  // thread 0 only
    const int pj = j0 + st * PB_KP;
    const int np = min(PB_KP, j1 - pj);
    fence_proxy_async();
    bulk_load(ring + (st % PB_NSTG) * PB_KP * pairc, corr + (int64_t)pj * pairc, np * pair_bytes,
              bars + st % PB_NSTG);
  };
  if (nst > 0) {
    if (T == 0) {
#pragma unroll
      for (int i = 0; i < PB_NSTG; ++i) mbar_init(bars + i, 1);
      mbar_init_fence();
      for (int st = 0; st < PB_NSTG - 1 && st < nst; ++st) issue(st);
    }
    __syncthreads();  // the barriers are initialised before anyone waits on them
  }
  const int npair = j1 - j0;
  const cx<R>* summ_c = summ + col * cs_summ;
  int src_nxt = lane < npair ? nsrc[j0 + lane] : 0, src_cur = 0;
  cx<R> acc[NREC / 2];
  interp_group<R, P>(grids + col * cs_grid, base, L, dL, t * q + a, med, h, n1, n2, acc);
  if (nst > 0) {
    const int set = h ? 2 : med;
    const bool neg = h && med;
    if (neg)
#pragma unroll
      for (int c = 0; c < NREC / 2; ++c) acc[c] = -acc[c];
    NearAcc<R> na;
    na.begin(acc);
    int st = 0;
    bool ok = true;
    for (; st < nst; ++st) {
      // slot (st - 1) % PB_NSTG was released by every thread at the barrier ending stage st - 1
      if (T == 0 && st + PB_NSTG - 1 < nst) issue(st + PB_NSTG - 1);
      const bool here = __all_sync(0xffffffffu, mbar_wait(bars + st % PB_NSTG, (st / PB_NSTG) & 1));
      if (here) {
        const cx<R>* rs = ring + (st % PB_NSTG) * PB_KP * pairc + (a * 2 + med) * NCORR;
#pragma unroll
        for (int k = 0; k < PB_KP; ++k) {
          const int jj = st * PB_KP + k;
          if (jj < npair) {
            if ((jj & 31) == 0) {
              src_cur = src_nxt;
              src_nxt = jj + 32 + lane < npair ? nsrc[j0 + jj + 32 + lane] : 0;
            }
            const int64_t sj = __shfl_sync(0xffffffffu, src_cur, jj & 31);
            cx<R> d[NCORR], sv[4];
            load_group(summ_c + (3 * sj + set) * 4, sv);
#pragma unroll
            for (int c = 0; c < NCORR; c += 2) load_pair_smem(rs + k * pairc + c, d + c);
            na.add(d, sv);
          }
        }
      }
      ok = __syncthreads_and(here) != 0;
      if (!ok) break;
    }
    if (!ok && T == 0) {
      // stages st .. min(st + PB_NSTG - 1, nst - 1) may still be in flight: let them land
      for (int s2 = st; s2 < nst && s2 < st + PB_NSTG; ++s2)
        (void)mbar_wait(bars + s2 % PB_NSTG, (s2 / PB_NSTG) & 1);
      atomicOr(tmo, 1);
    }
    na.end(acc);
    if (neg)
#pragma unroll
      for (int c = 0; c < NREC / 2; ++c) acc[c] = -acc[c];
  }
  // the ring is dead from here on: every thread passed the last stage's barrier
  if (act) {
    cx<R>* o = area + (int64_t)col * pb_col_complex(q) + (a * 2 + med) * NREC + 10 * h;
#pragma unroll
    for (int c = 0; c < NREC / 2; ++c) o[c] = acc[c];
  }
  __syncthreads();
  if (T < ncol * 3 * q) {
    const int c2 = T / (3 * q), r = T - c2 * 3 * q;
    const int kk = r / q, pa = r - kk * q;
    cx<R>* ar = area + (int64_t)c2 * pb_col_complex(q);
    cx<R> o[4];
    test_point(ar + pa * 2 * NREC, summ + c2 * cs_summ, tri, tp, sig, t, kk, pa, q, ke, ki, ze, zi, o);
    cx<R>* d = ar + 2 * q * NREC + (kk * q + pa) * 4;
#pragma unroll
    for (int c = 0; c < 4; ++c) d[c] = o[c];
  }
  __syncthreads();
  for (int u = T; u < ncol * 12; u += blockDim.x) {  // more tasks than threads when q = 1
    const int c2 = u / 12, r = u - c2 * 12;
    const int kk = r >> 2, c = r & 3;
    const cx<R>* sp = area + (int64_t)c2 * pb_col_complex(q) + 2 * q * NREC + kk * q * 4 + c;
    cx<R> v = czero<R>();
    for (int pa = 0; pa < q; ++pa) v += sp[pa * 4];
    const int row = valrow[(t * 3 + kk) * 4 + c];
    if (row >= 0) {
      cx<R>* yc = y + c2 * ldy;
      atomicAdd(&yc[row].re, v.re);
      atomicAdd(&yc[row].im, v.im);
    }
  }
}

// ================================================================ transposed apply
// x_bar = A^T y_bar: the stages of the apply in reverse order, each the
// transpose of its forward map (no conjugation):
//   T1 k_points_adj   rows -> tested values -> record adjoints at every point
//                     (Eqs. 1-3, 13, 14 testing transposed) and the
//                     triangle's own side-limit terms -> its summary adjoints
//   T2 k_near_adj_*   record adjoints of the targets -> summary adjoints of
//                     the source triangles (near records transposed): per
//                     pair over each target's record run, then per source
//                     over its reverse pair list (no atomics)
//   T3 k_interp_adj   record adjoints -> 16 grid fields (value and derivative
//                     stencils transposed), as a gather over covered points
//   T4 fft_conv(adjoint): each field with its medium's Green function
//   T5 k_proj_adj     grid -> point-source adjoints (value stencils
//                     transposed) -> summary adjoints (source expansion
//                     transposed), plus T1 + T2
//   T6 k_x_adj        summary adjoints -> unknowns (current expansion transposed)

// T1: one warp per triangle t.  Phase 1, lane (kk, a): the adjoints of the
// point-a quantities that the tested values of local edge kk read
// (u_type = w * ybar of the row, X = X_kk):
//   WE: X u0, wE: divX u0, WH: X (u1 + u2), wH: divX (u1 + u2),
//   E_e: -sg (n x X) u2, E_i: -sg X u3,
//   J_e + J_i: (n x X) u2 / 2 + X u3, M: sg (-X u2 + (n x X) u3) / 2.
// Phase 2, lane (a, medium, group): summed over kk, mapped to the 10 record
// values of the group (the transposes of medium_fields' combinations).
// Phase 3, lane (set, a | beta component): the own-summary adjoints summed
// over the points.
template <typename R>
__global__ void __launch_bounds__(PT_WARPS * 32)
    k_points_adj(const cx<R>* __restrict__ ybar, const int32_t* __restrict__ valrow, const double* __restrict__ tri,
                 const R* __restrict__ tp, const R* __restrict__ sig, int64_t nt, int q, R ke, R ki, R ze, R zi,
                 cx<R>* __restrict__ recb, cx<R>* __restrict__ sdir) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NA = 20;  // adjoint quantities per (kk, point)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * PT_WARPS + warp;
  if (t >= nt) return;
  cx<R>* part = reinterpret_cast<cx<R>*>(smem_raw) + (int64_t)warp * 3 * q * NA;  // [kk][a][NA]
  const double* g = tri + 16 * t;
  const R nrm[3] = {(R)g[12], (R)g[13], (R)g[14]};
  if (lane < 3 * q) {
    const int kk = lane / q, pa = lane - kk * q;
    const int64_t Qa = t * q + pa;
    const R* tq = tp + 16 * Qa;
    const R w = tq[3], sg = sig[Qa], divX = tq[13 + kk];
    const R X[3] = {tq[4 + 3 * kk], tq[5 + 3 * kk], tq[6 + 3 * kk]};
    const R nX[3] = {nrm[1] * X[2] - nrm[2] * X[1], nrm[2] * X[0] - nrm[0] * X[2], nrm[0] * X[1] - nrm[1] * X[0]};
    cx<R> u[4];
#pragma unroll
    for (int ty = 0; ty < 4; ++ty) {
      const int row = valrow[(t * 3 + kk) * 4 + ty];
      u[ty] = row >= 0 ? w * ybar[row] : czero<R>();
    }
    const cx<R> u12 = u[1] + u[2];
    cx<R>* o = part + (int64_t)(kk * q + pa) * NA;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      o[c] = X[c] * u[0];
      o[4 + c] = X[c] * u12;
      o[8 + c] = (-sg * nX[c]) * u[2];
      o[11 + c] = (-sg * X[c]) * u[3];
      o[14 + c] = (R(0.5) * nX[c]) * u[2] + X[c] * u[3];
      o[17 + c] = (R(0.5) * sg) * (nX[c] * u[3] - X[c] * u[2]);
    }
    o[3] = divX * u[0];
    o[7] = divX * u12;
  }
  __syncwarp();
  if (lane < 4 * q) {
    const int pa = lane >> 2, m = (lane >> 1) & 1, h = lane & 1;
    cx<R> ag[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) ag[i] = czero<R>();
    for (int kk = 0; kk < 3; ++kk) {
      const cx<R>* o = part + (int64_t)(kk * q + pa) * NA;
#pragma unroll
      for (int i = 0; i < 14; ++i) ag[i] += o[i];
    }
    const R k = m ? ki : ke, z = m ? zi : ze, sgm = m ? R(-1) : R(1);
    const cx<R>* Eb = ag + (m ? 11 : 8);
    cx<R> r[10];
    if (h == 0) {  // A, phi, grad phi, curl A
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        r[c] = (sgm * (-z * k)) * mulj(ag[c]) + (-z * k) * mulj(Eb[c]);
        r[4 + c] = (-z / k) * mulj(Eb[c]);
        r[7 + c] = sgm * ag[4 + c];
      }
      r[3] = (sgm * z / k) * mulj(ag[3]);
    } else {  // F, psi, grad psi (unused by the rows), curl F
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        r[c] = (-sgm * k / z) * mulj(ag[4 + c]);
        r[4 + c] = czero<R>();
        r[7 + c] = -(sgm * ag[c]) - Eb[c];
      }
      r[3] = (sgm / (k * z)) * mulj(ag[7]);
    }
    cx<R>* dst = recb + ((t * q + pa) * 2 + m) * NREC + 10 * h;
#pragma unroll
    for (int c = 0; c < 10; ++c) dst[c] = r[c];
  }
  __syncwarp();
  if (lane < 12) {
    const int set = lane >> 2, comp = lane & 3;
    const int base = set < 2 ? 14 : 17;  // J_e + J_i feeds sets 0 and 1, M set 2
    cx<R> acc = czero<R>();
    for (int pa = 0; pa < q; ++pa) {
      cx<R> v[3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        v[c] = part[(0 * q + pa) * NA + base + c] + part[(1 * q + pa) * NA + base + c] +
               part[(2 * q + pa) * NA + base + c];
      const R* tq = tp + 16 * (t * q + pa);
      if (comp == 0)
        acc += tq[0] * v[0] + tq[1] * v[1] + tq[2] * v[2];  // a: J = a (r - c) - beta
      else
        acc -= v[comp - 1];
    }
    sdir[(t * 3 + set) * 4 + comp] = acc;
  }
}

// T2a: one warp per target triangle t over its own near pairs (one
// contiguous run of records).  The pairs stream through a per-warp ring of
// NA_NSTG stages of NA_KP pairs (one bulk copy per pair into a slot padded to
// na_slot(q) complex values, so that the 16 (pair, point, medium) rows a warp
// load touches fall in distinct banks; bounded waits).  The target's record
// adjoints (q points x 2 media x 20) sit in shared memory.  Lane (pair k,
// point half ah, medium m, group h) forms, for pair k of the stage, the
// transpose of near_part summed over its points a = ah, ah + NA_AH, ...:
//   a_bar = sum_a r . dP1 + 2 phi_r dP0 + 2 grad_r . dQ + curl_r . dC,
//   beta_bar = sum_a -A_r dP0 - (the dQ x beta term transposed);
// the point halves are summed by one xor shuffle, and the pair's 12
// contributions are the per-set values J_e = (exterior, J), J_i = (interior,
// J), M = (exterior, M) - (interior, M).
constexpr int NA_AH = 2;  // lanes sharing one pair's points (1 or 2)
constexpr int NA_KP = 8 / NA_AH;
constexpr int NA_NSTG = 2;
__host__ __device__ __forceinline__ int na_slot(int q) {
  const int pc = NCORR * 2 * q;
  return pc + (((2 * NA_AH - pc) % 16) + 16) % 16;
}
__host__ __device__ __forceinline__ int na_warp_cx(int q) { return NA_NSTG * NA_KP * na_slot(q) + 40 * q; }
template <typename R>
__global__ void __launch_bounds__(PT_WARPS * 32, 4)
    k_near_adj_pairs(const cx<R>* __restrict__ corr, const int32_t* __restrict__ noff, const cx<R>* __restrict__ recb,
                     int64_t nt, int q, cx<R>* __restrict__ contrib, int* __restrict__ tmo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * PT_WARPS + warp;
  if (t >= nt) return;  // whole warp
  const int pairc = NCORR * 2 * q, slot = na_slot(q), wcx = na_warp_cx(q);
  cx<R>* ring = reinterpret_cast<cx<R>*>(smem_raw) + (int64_t)warp * wcx;
  cx<R>* rt = ring + NA_NSTG * NA_KP * slot;
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<cx<R>*>(smem_raw) + PT_WARPS * wcx) + warp * NA_NSTG;
  const int j0 = noff[t], j1 = noff[t + 1];
  const int nst = (j1 - j0 + NA_KP - 1) / NA_KP;
  if (nst == 0) return;
  const unsigned pair_bytes = (unsigned)(pairc * sizeof(cx<R>));
  auto issue = [&](int st) {
    const int pj = j0 + st * NA_KP;
    const int np = min(NA_KP, j1 - pj);
    uint64_t* b = bars + st % NA_NSTG;
    fence_proxy_async();
    mbar_expect_tx(b, np * pair_bytes);
    for (int k = 0; k < np; ++k)
      bulk_copy(ring + ((st % NA_NSTG) * NA_KP + k) * slot, corr + (int64_t)(pj + k) * pairc, pair_bytes, b);
  };
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NA_NSTG; ++i) mbar_init(bars + i, 1);
    mbar_init_fence();
    for (int st = 0; st < NA_NSTG - 1 && st < nst; ++st) issue(st);
  }
  {
    const cx<R>* rs = recb + t * q * 40;
    for (int u = lane; u < 40 * q; u += 32) rt[u] = rs[u];
  }
  __syncwarp();
  const int k = lane / (4 * NA_AH), ah = (lane >> 2) & (NA_AH - 1), m = (lane >> 1) & 1, h = lane & 1;
  const cx<R>* rl = rt + m * NREC + 10 * h;
  int st = 0;
  bool ok = true;
  for (; st < nst; ++st) {
    if (lane == 0 && st + NA_NSTG - 1 < nst) issue(st + NA_NSTG - 1);
    ok = __all_sync(0xffffffffu, mbar_wait(bars + st % NA_NSTG, (st / NA_NSTG) & 1));
    if (!ok) break;
    const int j = j0 + st * NA_KP + k;
    const cx<R>* dp = ring + ((st % NA_NSTG) * NA_KP + k) * slot + m * NCORR;
    cx<R> al = czero<R>(), be[3] = {czero<R>(), czero<R>(), czero<R>()};
    if (j < j1) {
      for (int a = ah; a < q; a += NA_AH) {
        cx<R> r[10], d[NCORR];
#pragma unroll
        for (int c = 0; c < 10; c += 2) load_pair_smem(rl + a * 40 + c, r + c);
#pragma unroll
        for (int c = 0; c < NCORR; c += 2) load_pair_smem(dp + a * 2 * NCORR + c, d + c);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          cfma(al, r[c], d[1 + c]);
          cfma(al, R(2) * r[4 + c], d[4 + c]);
          cfma(al, r[7 + c], d[7 + c]);
          be[c] -= r[c] * d[0];
        }
        cfma(al, R(2) * r[3], d[0]);
        be[0] += r[9] * d[5] - r[8] * d[6];
        be[1] += r[7] * d[6] - r[9] * d[4];
        be[2] += r[8] * d[4] - r[7] * d[5];
      }
    }
    cx<R> v[4] = {al, be[0], be[1], be[2]};
    if (NA_AH == 2)  // the two point halves (lane bit 2)
#pragma unroll
      for (int c = 0; c < 4; ++c)
        v[c] += mk(__shfl_xor_sync(0xffffffffu, v[c].re, 4), __shfl_xor_sync(0xffffffffu, v[c].im, 4));
    // (exterior, M) - (interior, M): lanes h = 1 differ in bit 1 (medium)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const cx<R> o = mk(__shfl_xor_sync(0xffffffffu, v[c].re, 2), __shfl_xor_sync(0xffffffffu, v[c].im, 2));
      if (h) v[c] -= o;
    }
    if (j < j1 && ah == 0 && (h == 0 || m == 0)) {
      cx<R>* cj = contrib + (int64_t)j * 12 + (h ? 8 : 4 * m);
#pragma unroll
      for (int c = 0; c < 4; ++c) cj[c] = v[c];
    }
    __syncwarp();
  }
  if (!ok) {
    for (int s2 = st; s2 < nst && s2 < st + NA_NSTG; ++s2) (void)mbar_wait(bars + s2 % NA_NSTG, (s2 / NA_NSTG) & 1);
    if (lane == 0) atomicOr(tmo, 1);
  }
}

// T2b: thread per (source triangle s, set, component): sdir plus the pair
// contributions of the pairs whose source is s, in reverse-list order.
template <typename R>
__global__ void k_near_adj_sum(const int32_t* __restrict__ roff, const int32_t* __restrict__ rpair,
                               const cx<R>* __restrict__ contrib, const cx<R>* __restrict__ sdir, int64_t nt,
                               cx<R>* __restrict__ snear) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nt * 12) return;
  const int64_t sidx = idx / 12;
  const int c = (int)(idx - sidx * 12);
  cx<R> acc = sdir[idx];
  for (int rp = roff[sidx]; rp < roff[sidx + 1]; ++rp) acc += contrib[(int64_t)rpair[rp] * 12 + c];
  snear[idx] = acc;
}

// T3: one warp per covered grid point i.  Lane pr < 20 reads the 16-byte
// portion pr of the 320-byte record-adjoint row of every entry of the point
// (records 2 pr, 2 pr + 1 of the 40 = 2 media x 2 groups x 10; one coalesced
// row per load instruction, IADJ_INFLIGHT rows in flight) and accumulates
// each record against all four entry weights (value W, derivatives Wx, Wy,
// Wz).  The transposed interpolation of one group (records r0..r9) is then a
// fixed combination of those sums:
//   f0 = W r0 + Wz r8 - Wy r9,  f1 = W r1 - Wz r7 + Wx r9,
//   f2 = W r2 + Wy r7 - Wx r8,  f3 = W r3 + Wx r4 + Wy r5 + Wz r6,
// formed by lanes 0..15 (group g4, field f) and written field-major.
constexpr int IADJ_INFLIGHT = 4;
template <typename R>
__global__ void __launch_bounds__(256) k_interp_adj(const cx<R>* __restrict__ recb, const int32_t* __restrict__ gpt,
                                                    const int32_t* __restrict__ goff, const int32_t* __restrict__ gq,
                                                    const R* __restrict__ gw, const R* __restrict__ gd,
                                                    int64_t ngnz, int64_t ng, cx<R>* __restrict__ grids) {
  __shared__ cx<R> red[8][20][8];  // [warp in CTA][portion][record k * 4 + weight]
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const bool act = lane < 20 && i < ngnz;
  cx<R> acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = czero<R>();
  if (act) {
    const int e1 = goff[i + 1];
    for (int e = goff[i]; e < e1; e += IADJ_INFLIGHT) {
      int qe[IADJ_INFLIGHT];
      R w[IADJ_INFLIGHT][4];
#pragma unroll
      for (int u = 0; u < IADJ_INFLIGHT; ++u) {
        const int eu = e + u < e1 ? e + u : e;
        const R on = e + u < e1 ? R(1) : R(0);
        qe[u] = gq[eu];
        w[u][0] = on * gw[eu];
#pragma unroll
        for (int c = 0; c < 3; ++c) w[u][1 + c] = on * gd[3 * (int64_t)eu + c];
      }
      cx<R> v[IADJ_INFLIGHT][2];
#pragma unroll
      for (int u = 0; u < IADJ_INFLIGHT; ++u) load_pair(recb + (int64_t)qe[u] * (2 * NREC) + 2 * lane, v[u]);
#pragma unroll
      for (int u = 0; u < IADJ_INFLIGHT; ++u)
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
          for (int c = 0; c < 4; ++c) axpy2(acc[k * 4 + c], w[u][c], v[u][k]);
    }
  }
  if (lane < 20)
#pragma unroll
    for (int c = 0; c < 8; ++c) red[wl][lane][c] = acc[c];
  __syncwarp();
  if (lane < 16 && i < ngnz) {
    // record 10 h + r of group g4 = 2 m + h sits in portion 5 g4 + r / 2,
    // slot (r & 1) * 4 + weight; weights 0 W, 1 Wx, 2 Wy, 3 Wz
    const int g4 = lane >> 2, f = lane & 3;
    const cx<R>(*rp)[8] = red[wl] + 5 * g4;
#define RW(r, wt) rp[(r) >> 1][((r) & 1) * 4 + (wt)]
    cx<R> o;
    switch (f) {
      case 0: o = RW(0, 0) + RW(8, 3) - RW(9, 2); break;
      case 1: o = RW(1, 0) - RW(7, 3) + RW(9, 1); break;
      case 2: o = RW(2, 0) + RW(7, 2) - RW(8, 1); break;
      default: o = RW(3, 0) + RW(4, 1) + RW(5, 2) + RW(6, 3); break;
    }
#undef RW
    grids[(int64_t)lane * ng + gpt[i]] = o;
  }
}

// T5: one warp per triangle t; lane (point a, set): the transposed value
// interpolation of the convolved adjoint grid (point-major; J_e from fields
// 0..3, J_i from 8..11, M from 4..7 minus 12..15), then the transposed point
// sources (a_bar += w (r - c) . qb + 2 w qb_div, beta_bar -= w qb), summed
// over the points in point order and added to snear.
template <typename R, int P>
__global__ void __launch_bounds__(PT_WARPS * 32)
    k_proj_adj(const cx<R>* __restrict__ grids, const int32_t* __restrict__ base, const R* __restrict__ L,
               const R* __restrict__ tp, const cx<R>* __restrict__ snear, int64_t nt, int q, int n1, int n2,
               cx<R>* __restrict__ stot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * PT_WARPS + warp;
  if (t >= nt) return;
  cx<R>* red = reinterpret_cast<cx<R>*>(smem_raw) + (int64_t)warp * 32 * 4;  // [lane][4]
  if (lane < 3 * q) {
    const int pa = lane / 3, set = lane - pa * 3;
    const int64_t Qi = t * q + pa;
    R Lx[P], Ly[P], Lz[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
      Lx[i] = L[(3 * Qi + 0) * P + i];
      Ly[i] = L[(3 * Qi + 1) * P + i];
      Lz[i] = L[(3 * Qi + 2) * P + i];
    }
    const int b0 = base[3 * Qi], b1 = base[3 * Qi + 1], b2 = base[3 * Qi + 2];
    const int fa = set == 0 ? 0 : (set == 1 ? 8 : 4);
    cx<R> qb[4] = {czero<R>(), czero<R>(), czero<R>(), czero<R>()};
#pragma unroll
    for (int i = 0; i < P; ++i)
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const R wxy = Lx[i] * Ly[j];
        const int64_t rowi = ((int64_t)(b0 + i) * n1 + (b1 + j)) * n2 + b2;
#pragma unroll
        for (int k = 0; k < P; ++k) {
          const R W = wxy * Lz[k];
          cx<R> gv[4];
          load_group(grids + (rowi + k) * NFIELD_OUT + fa, gv);
          if (set == 2) {
            cx<R> gi[4];
            load_group(grids + (rowi + k) * NFIELD_OUT + 12, gi);
#pragma unroll
            for (int f = 0; f < 4; ++f) gv[f] -= gi[f];
          }
#pragma unroll
          for (int f = 0; f < 4; ++f) axpy(qb[f], W, gv[f]);
        }
      }
    const R* tq = tp + 16 * Qi;
    const R w = tq[3];
    red[lane * 4 + 0] = w * (tq[0] * qb[0] + tq[1] * qb[1] + tq[2] * qb[2]) + (R(2) * w) * qb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) red[lane * 4 + 1 + c] = -(w * qb[c]);
  }
  __syncwarp();
  if (lane < 12) {
    const int set = lane >> 2, comp = lane & 3;
    cx<R> acc = snear[(t * 3 + set) * 4 + comp];
    for (int pa = 0; pa < q; ++pa) acc += red[(pa * 3 + set) * 4 + comp];
    stot[(t * 3 + set) * 4 + comp] = acc;
  }
}

// T6: thread per unknown: x_bar = sum over its uses (triangle t, local edge k,
// set, sign) of sign cX_k (a_bar + (v_k - c) . beta_bar).
template <typename R>
__global__ void k_x_adj(const cx<R>* __restrict__ stot, const int32_t* __restrict__ xsrc,
                        const double* __restrict__ tri, const double* __restrict__ cX, int64_t N,
                        cx<R>* __restrict__ xbar) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  cx<R> acc = czero<R>();
  for (int u = 0; u < 4; ++u) {
    const int32_t code = xsrc[4 * i + u];
    if (code == 0) break;
    const int64_t c = (code > 0 ? code : -code) - 1;
    const int set = (int)(c % 3);
    const int64_t tk = c / 3, t = tk / 3;
    const int k = (int)(tk - t * 3);
    const double* g = tri + 16 * t;
    const cx<R>* sb = stot + (t * 3 + set) * 4;
    cx<R> v = sb[0];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) v += (R)(g[3 * k + cc] - g[9 + cc]) * sb[1 + cc];
    const R f = (R)cX[3 * t + k] * (code > 0 ? R(1) : R(-1));
    acc += f * v;
  }
  xbar[i] = acc;
}

template <typename R>
using PointsFn = void (*)(const cx<R>*, const int32_t*, const R*, const R*, const cx<R>*, const int32_t*,
                          const int32_t*, const cx<R>*, const double*, const R*, const R*, int64_t, int, int, int,
                          int, R, R, R, R, int, const int32_t*, cx<R>*, int*, const cx<R>*, cx<R>*);

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
  k_sources<R><<<(int)cdiv(Q, 128), 128, 0, s>>>(x, op->unk, op->cX, op->tri, op->qp, op->qw, Q, op->q, pd.summ,
                                                 pd.qsrc, y, op->N, 0, 0);
  CK(cudaGetLastError());
  prof_mark(op, s);
  if (op->ngnz > 0) {
    k_gather<R><<<(int)cdiv(op->ngnz * 32, 256), 256, 0, s>>>(pd.qsrc, op->gpt, op->goff, op->gent,
                                                              gather_weights<R>(op), op->ngnz, ng, pd.src, 0, 0);
    CK(cudaGetLastError());
  }
  prof_mark(op, s);
  int rc = fft_conv<R>(op, pd, s, false);
  if (rc) return rc;
  prof_mark(op, s);
  {
    const size_t sm = pt_smem_bytes(op->q, sizeof(cx<R>));
    PointsFn<R> fn = op->q == 6 ? (op->p == 2 ? k_points<R, 2, false, 6> : op->p == 3 ? k_points<R, 3, false, 6>
                                                                                   : k_points<R, 4, false, 6>)
                                : (op->p == 2 ? k_points<R, 2> : op->p == 3 ? k_points<R, 3> : k_points<R, 4>);
    if (int rc_ = set_max_smem(op->device, (const void*)fn, (int)sm)) return rc_;
    fn<<<(int)cdiv(nt, PT_WARPS), PT_WARPS * 32, sm, s>>>(pd.grid, op->base, pd.L, pd.dL, pd.near, op->noff, op->nsrc, pd.summ,
                                                  op->tri, pd.tp, pd.sig, nt, op->q, n0, n1, n2, (R)op->ke, (R)op->ki,
                                                  (R)op->ze, (R)op->zi, op->npairs > 0 ? 1 : 0, op->valrow, y,
                                                  op->tmo_d, nullptr, nullptr);
    CK(cudaGetLastError());
  }
  prof_mark(op, s);
  return SCABEM_OK;
}

template <typename R>
using PointsBatchFn = void (*)(const cx<R>*, const int32_t*, const R*, const R*, const cx<R>*, const int32_t*,
                               const int32_t*, const cx<R>*, const double*, const R*, const R*, int64_t, int, int, int,
                               int, R, R, R, R, int, const int32_t*, cx<R>*, int*, int64_t, int64_t, int64_t, int);

template <typename R>
int apply_batch(scabem_op* op, const cx<R>* x, int64_t ldx, cx<R>* y, int64_t ldy, int k, cudaStream_t s) {
  PrecData<R>& pd = pdata<R>(op);
  if (k < 1 || k > KBATCH || k > pd.kcap) {
    set_error("apply_batch: batch size outside the workspace capacity");
    return SCABEM_E_ARG;
  }
  const int64_t nt = op->nt, Q = op->Q;
  const int n0 = op->n[0], n1 = op->n[1], n2 = op->n[2];
  const int64_t ng = (int64_t)n0 * n1 * n2;
  prof_mark(op, s);
  k_sources<R><<<dim3((unsigned)cdiv(Q, 128), k), 128, 0, s>>>(x, op->unk, op->cX, op->tri, op->qp, op->qw, Q,
                                                               op->q, pd.summ, pd.qsrc, y, op->N, ldx, ldy);
  CK(cudaGetLastError());
  prof_mark(op, s);
  if (op->ngnz > 0) {
    k_gather<R><<<dim3((unsigned)cdiv(op->ngnz * 32, 256), k), 256, 0, s>>>(
        pd.qsrc, op->gpt, op->goff, op->gent, gather_weights<R>(op), op->ngnz, ng, pd.src, col_stride_qsrc(op),
        col_stride_grid(op));
    CK(cudaGetLastError());
  }
  prof_mark(op, s);
  int rc = fft_conv<R>(op, pd, s, false, k);
  if (rc) return rc;
  prof_mark(op, s);
  {
    const size_t sm = pb_smem_bytes(op->q, k, sizeof(cx<R>));
    PointsBatchFn<R> fn =
        op->q == 6 ? (op->p == 2 ? k_points_batch<R, 2, 6> : op->p == 3 ? k_points_batch<R, 3, 6> : k_points_batch<R, 4, 6>)
                   : (op->p == 2 ? k_points_batch<R, 2> : op->p == 3 ? k_points_batch<R, 3> : k_points_batch<R, 4>);
    if (int rc_ = set_max_smem(op->device, (const void*)fn, (int)pb_smem_bytes(op->q, KBATCH, sizeof(cx<R>))))
      return rc_;
    fn<<<(unsigned)nt, pb_threads(op->q, k), sm, s>>>(
        pd.grid, op->base, pd.L, pd.dL, pd.near, op->noff, op->nsrc, pd.summ, op->tri, pd.tp, pd.sig, nt, op->q, n0,
        n1, n2, (R)op->ke, (R)op->ki, (R)op->ze, (R)op->zi, op->npairs > 0 ? 1 : 0, op->valrow, y, op->tmo_d,
        col_stride_grid(op), col_stride_summ(op), ldy, k);
    CK(cudaGetLastError());
  }
  prof_mark(op, s);
  return SCABEM_OK;
}

template <typename R>
using ProjAdjFn = void (*)(const cx<R>*, const int32_t*, const R*, const R*, const cx<R>*, int64_t, int, int, int,
                           cx<R>*);

// x_bar = A^T y_bar (one right-hand side), stages T1-T6.
template <typename R>
int apply_adjoint_one(scabem_op* op, const cx<R>* ybar, cx<R>* xbar, cudaStream_t s) {
  PrecData<R>& pd = pdata<R>(op);
  const int64_t nt = op->nt;
  const int q = op->q;
  const int64_t ng = (int64_t)op->n[0] * op->n[1] * op->n[2];
  cx<R>* sdir = pd.sbar;
  cx<R>* snear = pd.sbar + nt * 12;
  const int blocks = (int)cdiv(nt, PT_WARPS);
  {
    const size_t sm = (size_t)PT_WARPS * 3 * q * 20 * sizeof(cx<R>);
    if (int rc_ = set_max_smem(op->device, (const void*)k_points_adj<R>, (int)sm)) return rc_;
    k_points_adj<R><<<blocks, PT_WARPS * 32, sm, s>>>(ybar, op->valrow, op->tri, pd.tp, pd.sig, nt, q, (R)op->ke,
                                                      (R)op->ki, (R)op->ze, (R)op->zi, pd.recb, sdir);
    CK(cudaGetLastError());
  }
  const cx<R>* s_after_near = sdir;
  if (op->npairs > 0) {
    const size_t sm = (size_t)PT_WARPS * na_warp_cx(q) * sizeof(cx<R>) + (size_t)PT_WARPS * NA_NSTG * sizeof(uint64_t);
    if (int rc_ = set_max_smem(op->device, (const void*)k_near_adj_pairs<R>, (int)sm)) return rc_;
    k_near_adj_pairs<R><<<blocks, PT_WARPS * 32, sm, s>>>(pd.near, op->noff, pd.recb, nt, q, pd.nadj, op->tmo_d);
    CK(cudaGetLastError());
    k_near_adj_sum<R><<<(int)cdiv(nt * 12, 256), 256, 0, s>>>(op->roff, op->rpair, pd.nadj, sdir, nt, snear);
    CK(cudaGetLastError());
    s_after_near = snear;
  }
  if (op->ngnz > 0) {
    k_interp_adj<R><<<(int)cdiv(op->ngnz * 32, 256), 256, 0, s>>>(pd.recb, op->gpt, op->goff, op->gent,
                                                                 gather_weights<R>(op), gather_dweights<R>(op),
                                                                 op->ngnz, ng, pd.src);
    CK(cudaGetLastError());
  }
  int rc = fft_conv<R>(op, pd, s, true);
  if (rc) return rc;
  {
    const size_t sm = (size_t)PT_WARPS * 32 * 4 * sizeof(cx<R>);
    ProjAdjFn<R> fn = op->p == 2 ? k_proj_adj<R, 2> : op->p == 3 ? k_proj_adj<R, 3> : k_proj_adj<R, 4>;
    fn<<<blocks, PT_WARPS * 32, sm, s>>>(pd.grid, op->base, pd.L, pd.tp, s_after_near, nt, q, op->n[1], op->n[2],
                                         sdir);
    CK(cudaGetLastError());
  }
  k_x_adj<R><<<(int)cdiv(op->N, 256), 256, 0, s>>>(sdir, op->xsrc, op->tri, op->cX, op->N, xbar);
  CK(cudaGetLastError());
  return SCABEM_OK;
}

// hs[p] = d(lam^T A x)/d sigma_p [per S] at every quadrature point
// (complex128): the apply's stages up to the records, then the derivative
// of the sigma-weighted testing (k_points in its sensitivity mode).  yscr:
// N complex of scratch.
int sigma_sensitivity_op(scabem_op* op, const cx<double>* x, const cx<double>* lam, cx<double>* hs,
                         cx<double>* yscr, cudaStream_t s) {
  PrecData<double>& pd = op->d;
  const int64_t nt = op->nt, Q = op->Q;
  const int n0 = op->n[0], n1 = op->n[1], n2 = op->n[2];
  const int64_t ng = (int64_t)n0 * n1 * n2;
  k_sources<double><<<(int)cdiv(Q, 128), 128, 0, s>>>(x, op->unk, op->cX, op->tri, op->qp, op->qw, Q, op->q,
                                                      pd.summ, pd.qsrc, yscr, op->N, 0, 0);
  CK(cudaGetLastError());
  if (op->ngnz > 0) {
    k_gather<double><<<(int)cdiv(op->ngnz * 32, 256), 256, 0, s>>>(pd.qsrc, op->gpt, op->goff, op->gent, op->gwd,
                                                                   op->ngnz, ng, pd.src, 0, 0);
    CK(cudaGetLastError());
  }
  int rc = fft_conv<double>(op, pd, s, false);
  if (rc) return rc;
  const size_t sm = pt_smem_bytes(op->q, sizeof(cx<double>));
  PointsFn<double> fn = op->p == 2 ? k_points<double, 2, true> : op->p == 3 ? k_points<double, 3, true>
                                                                            : k_points<double, 4, true>;
  if (int rc_ = set_max_smem(op->device, (const void*)fn, (int)sm)) return rc_;
  fn<<<(int)cdiv(nt, PT_WARPS), PT_WARPS * 32, sm, s>>>(pd.grid, op->base, pd.L, pd.dL, pd.near, op->noff, op->nsrc,
                                                        pd.summ, op->tri, pd.tp, pd.sig, nt, op->q, n0, n1, n2, op->ke,
                                                        op->ki, op->ze, op->zi, op->npairs > 0 ? 1 : 0, op->valrow,
                                                        yscr, op->tmo_d, lam, hs);
  CK(cudaGetLastError());
  return SCABEM_OK;
}

int selftest_wait(scabem_op* op, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(op->tmo_d);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
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
template int apply_adjoint_one<float>(scabem_op*, const cx<float>*, cx<float>*, cudaStream_t);
template int apply_adjoint_one<double>(scabem_op*, const cx<double>*, cx<double>*, cudaStream_t);
template int apply_one<double>(scabem_op*, const cx<double>*, cx<double>*, cudaStream_t);
template int apply_batch<float>(scabem_op*, const cx<float>*, int64_t, cx<float>*, int64_t, int, cudaStream_t);
template int apply_batch<double>(scabem_op*, const cx<double>*, int64_t, cx<double>*, int64_t, int, cudaStream_t);
