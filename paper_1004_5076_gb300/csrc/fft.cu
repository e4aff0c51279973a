// Grid convolution by zero-padded 3-D FFT, fused with the Green's-function
// multiply (the FFT acceleration of Appendix B, on the uniform grid of the
// precorrected-FFT method).
//
// Layout: physical grids are [field][i0][i1][i2] with n0 x n1 x n2 points; the
// transform size is P = 2n per axis.  The convolution runs in three kernels:
//   stage A: forward FFT along axis 0 of the 12 source fields, input pruned
//            to i0 < n0, output [field][k0][i1][i2] (P0 x n1 x n2);
//   stage B: per k0 plane, forward 2-D FFT over (i1, i2) (input pruned to the
//            physical n1 x n2 corner), multiply by the Green spectrum of the
//            medium, inverse 2-D FFT, keep the physical corner: 12 -> 16 fields;
//   stage C: inverse FFT along axis 0, keep i0 < n0.
// Every FFT is a shared-memory Stockham transform (radix 8, then 4 or 2), one
// CTA owning whole lines, so each field makes one HBM round trip per stage.
// The 1/(P0 P1 P2) scale is folded into the stored spectra.
#include <cuda_runtime.h>

#include "common.cuh"

namespace {

template <typename R, int DIR>
__device__ __forceinline__ cx<R> rot(cx<R> a) {  // multiply by DIR * j
  return DIR < 0 ? mk(a.im, -a.re) : mk(-a.im, a.re);
}

template <typename R, int DIR>
__device__ __forceinline__ void dft2(cx<R>& a, cx<R>& b) {
  cx<R> t = a;
  a = t + b;
  b = t - b;
}

template <typename R, int DIR>
__device__ __forceinline__ void dft4(cx<R>& a0, cx<R>& a1, cx<R>& a2, cx<R>& a3) {
  cx<R> t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, u = rot<R, DIR>(a1 - a3);
  a0 = t0 + t2;
  a2 = t0 - t2;
  a1 = t1 + u;
  a3 = t1 - u;
}

template <typename R, int RAD, int DIR>
__device__ __forceinline__ void dft(cx<R>* v) {
  if constexpr (RAD == 2) {
    dft2<R, DIR>(v[0], v[1]);
  } else if constexpr (RAD == 4) {
    dft4<R, DIR>(v[0], v[1], v[2], v[3]);
  } else {
    // 8 = 2 x 4: even / odd 4-point transforms, then combine with w8^k
    cx<R> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    cx<R> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<R, DIR>(e0, e1, e2, e3);
    dft4<R, DIR>(o0, o1, o2, o3);
    const R s = R(0.70710678118654752440);
    // w8^1 = (1 + DIR j)/sqrt2, w8^2 = DIR j, w8^3 = (-1 + DIR j)/sqrt2
    cx<R> w1 = s * (o1 + rot<R, DIR>(o1));
    cx<R> w2 = rot<R, DIR>(o2);
    cx<R> w3 = s * (rot<R, DIR>(o3) - o3);
    v[0] = e0 + o0;
    v[4] = e0 - o0;
    v[1] = e1 + w1;
    v[5] = e1 - w1;
    v[2] = e2 + w2;
    v[6] = e2 - w2;
    v[3] = e3 + w3;
    v[7] = e3 - w3;
  }
}

// One out-of-place Stockham pass over `nlines` lines of length `len`.
// Element j of line l lives at buf[l*ls + j*es].  Ns = product of the radices
// of the previous passes.  JFAST maps consecutive threads to consecutive j
// (for contiguous lines); otherwise to consecutive lines.
template <typename R, int RAD, int DIR, bool JFAST>
__device__ __forceinline__ void pass(const cx<R>* __restrict__ src, cx<R>* __restrict__ dst, int len, int Ns,
                                     int nlines, int ls, int es, const cx<R>* __restrict__ tw) {
  const int per = len / RAD;
  const int nb = nlines * per;
  const int ts = len / (Ns * RAD);
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    int line, j;
    if (JFAST) {
      j = b % per;
      line = b / per;
    } else {
      line = b % nlines;
      j = b / nlines;
    }
    const cx<R>* s = src + (int64_t)line * ls;
    cx<R>* d = dst + (int64_t)line * ls;
    const int k = j % Ns;
    cx<R> v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = s[(j + r * per) * es];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        cx<R> t = tw[r * k * ts];
        if (DIR > 0) t = conj(t);
        v[r] = v[r] * t;
      }
    }
    dft<R, RAD, DIR>(v);
    const int o = (j / Ns) * Ns * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) d[(o + r * Ns) * es] = v[r];
  }
}

// Full FFT of nlines lines, ping-ponging between b0 (input) and b1.  Returns
// the buffer that holds the result.  All threads of the block must call it.
template <typename R, int DIR, bool JFAST>
__device__ cx<R>* fft_lines(cx<R>* b0, cx<R>* b1, int len, int nlines, int ls, int es, const cx<R>* tw) {
  cx<R>* in = b0;
  cx<R>* out = b1;
  int Ns = 1;
  while (Ns < len) {
    const int rem = len / Ns;
    if (rem >= 8) {
      pass<R, 8, DIR, JFAST>(in, out, len, Ns, nlines, ls, es, tw);
      Ns *= 8;
    } else if (rem == 4) {
      pass<R, 4, DIR, JFAST>(in, out, len, Ns, nlines, ls, es, tw);
      Ns *= 4;
    } else {
      pass<R, 2, DIR, JFAST>(in, out, len, Ns, nlines, ls, es, tw);
      Ns *= 2;
    }
    __syncthreads();
    cx<R>* t = in;
    in = out;
    out = t;
  }
  return in;
}

// ---------------------------------------------------------------- stage A / C
// Columns c in [0, C) of the [field][i0][c] layout; one CTA owns CB columns
// of one field over the whole axis 0.
template <typename R, int DIR>
__global__ void k_axis0(const cx<R>* __restrict__ in, cx<R>* __restrict__ out, int n_in, int n_out, int P0, int C,
                        int CB, const cx<R>* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  cx<R>* b0 = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* b1 = b0 + P0 * CB;
  const int f = blockIdx.y;
  const int c0 = blockIdx.x * CB;
  const int64_t fin = (int64_t)f * n_in * C;
  for (int idx = threadIdx.x; idx < P0 * CB; idx += blockDim.x) {
    const int i0 = idx / CB, l = idx - (idx / CB) * CB;
    cx<R> v = czero<R>();
    if (i0 < n_in && c0 + l < C) v = in[fin + (int64_t)i0 * C + c0 + l];
    b0[idx] = v;
  }
  __syncthreads();
  cx<R>* res = fft_lines<R, DIR, false>(b0, b1, P0, CB, 1, CB, tw);
  const int64_t fout = (int64_t)f * n_out * C;
  for (int idx = threadIdx.x; idx < n_out * CB; idx += blockDim.x) {
    const int k0 = idx / CB, l = idx - (idx / CB) * CB;
    if (c0 + l < C) out[fout + (int64_t)k0 * C + c0 + l] = res[idx];
  }
}

// ---------------------------------------------------------------- stage B
// One CTA per (k0 plane, source field).  Source fields:
//   0..3  exterior J (x, y, z, div)  -> outputs 0..3 with G_e
//   4..7  interior J                 -> outputs 8..11 with G_i
//   8..11 exterior M                 -> outputs 4..7 with G_e and 12..15 with -G_i
template <typename R>
__global__ void k_planes(const cx<R>* __restrict__ A, cx<R>* __restrict__ B, const cx<R>* __restrict__ ghE,
                         const cx<R>* __restrict__ ghI, int P0, int n1, int n2, int P1, int P2,
                         const cx<R>* __restrict__ tw1, const cx<R>* __restrict__ tw2) {
  extern __shared__ unsigned char smem_raw[];
  const int plane = P1 * P2;
  cx<R>* X = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* Y = X + plane;
  cx<R>* Z = Y + plane;
  const int k0 = blockIdx.x;
  const int f = blockIdx.y;
  const int64_t C = (int64_t)n1 * n2;
  const cx<R>* src = A + ((int64_t)f * P0 + k0) * C;
  for (int idx = threadIdx.x; idx < plane; idx += blockDim.x) {
    const int i1 = idx / P2, i2 = idx - (idx / P2) * P2;
    cx<R> v = czero<R>();
    if (i1 < n1 && i2 < n2) v = src[i1 * n2 + i2];
    X[idx] = v;
    Y[idx] = czero<R>();
  }
  __syncthreads();
  // rows (axis 2), only the n1 non-zero rows
  cx<R>* r = fft_lines<R, -1, true>(X, Y, P2, n1, P2, 1, tw2);
  cx<R>* o = (r == X) ? Y : X;
  // columns (axis 1), all P2 of them
  cx<R>* S = fft_lines<R, -1, false>(r, o, P1, P2, 1, P2, tw1);
  cx<R>* T = (S == X) ? Y : X;  // free buffer besides Z

  const int h0 = P0 / 2 + 1, h1 = P1 / 2 + 1, h2 = P2 / 2 + 1;
  const int q0 = min(k0, P0 - k0);
  int nout = (f >= 8) ? 2 : 1;
  for (int which = 0; which < nout; ++which) {
    int fo;
    const cx<R>* gh;
    R sgn = R(1);
    if (f < 4) {
      fo = f;
      gh = ghE;
    } else if (f < 8) {
      fo = 8 + (f - 4);
      gh = ghI;
    } else if (which == 0) {
      fo = 4 + (f - 8);
      gh = ghE;
    } else {
      fo = 12 + (f - 8);
      gh = ghI;
      sgn = R(-1);
    }
    const cx<R>* g0 = gh + (int64_t)q0 * h1 * h2;
    for (int idx = threadIdx.x; idx < plane; idx += blockDim.x) {
      const int k1 = idx / P2, k2 = idx - (idx / P2) * P2;
      const int q1 = min(k1, P1 - k1), q2 = min(k2, P2 - k2);
      Z[idx] = sgn * (S[idx] * g0[q1 * h2 + q2]);
    }
    __syncthreads();
    cx<R>* u = fft_lines<R, 1, false>(Z, T, P1, P2, 1, P2, tw1);
    cx<R>* w = (u == Z) ? T : Z;
    cx<R>* v = fft_lines<R, 1, true>(u, w, P2, n1, P2, 1, tw2);
    cx<R>* dst = B + ((int64_t)fo * P0 + k0) * C;
    for (int idx = threadIdx.x; idx < n1 * n2; idx += blockDim.x) {
      const int i1 = idx / n2, i2 = idx - (idx / n2) * n2;
      dst[idx] = v[i1 * P2 + i2];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- generic 3-D FFT (set-up)
template <typename R, int DIR>
__global__ void k_fft_axis(cx<R>* data, int len, int inner, int64_t nlines, int CB, const cx<R>* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  cx<R>* b0 = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* b1 = b0 + len * CB;
  const int64_t L0 = (int64_t)blockIdx.x * CB;
  for (int idx = threadIdx.x; idx < len * CB; idx += blockDim.x) {
    const int j = idx / CB, l = idx - (idx / CB) * CB;
    const int64_t L = L0 + l;
    cx<R> v = czero<R>();
    if (L < nlines) v = data[(L / inner) * ((int64_t)len * inner) + (L % inner) + (int64_t)j * inner];
    b0[idx] = v;
  }
  __syncthreads();
  cx<R>* res = fft_lines<R, DIR, false>(b0, b1, len, CB, 1, CB, tw);
  for (int idx = threadIdx.x; idx < len * CB; idx += blockDim.x) {
    const int j = idx / CB, l = idx - (idx / CB) * CB;
    const int64_t L = L0 + l;
    if (L < nlines) data[(L / inner) * ((int64_t)len * inner) + (L % inner) + (int64_t)j * inner] = res[idx];
  }
}

template <typename R>
__global__ void k_twiddles(cx<R>* tw, int len) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= len) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)len, &s, &c);
  tw[m] = mk(R(c), R(-s));
}

template <typename R>
int cb_for(int len) {
  // lines per CTA so that two buffers stay within ~96 KB (c64) / 128 KB (c128)
  int budget = (sizeof(R) == 4) ? 96 * 1024 : 128 * 1024;
  int cb = budget / (2 * len * (int)sizeof(cx<R>));
  if (cb > 32) cb = 32;
  if (cb < 1) cb = 1;
  return cb;
}

}  // namespace

template <typename R>
int make_twiddles(cx<R>* tw, int len, cudaStream_t s) {
  k_twiddles<R><<<(int)cdiv(len, 256), 256, 0, s>>>(tw, len);
  CK(cudaGetLastError());
  return SCABEM_OK;
}

template <typename R>
int fft3d_full(scabem_op* op, cx<R>* data, const cx<R>* const tw[3], int dir, cudaStream_t s) {
  const int64_t total = (int64_t)op->P[0] * op->P[1] * op->P[2];
  for (int a = 0; a < 3; ++a) {
    const int len = op->P[a];
    int inner = 1;
    for (int b = a + 1; b < 3; ++b) inner *= op->P[b];
    const int64_t nlines = total / len;
    const int cb = cb_for<R>(len);
    const size_t sm = 2 * (size_t)len * cb * sizeof(cx<R>);
    const int blocks = (int)cdiv(nlines, cb);
    if (dir < 0) {
      CK(cudaFuncSetAttribute(k_fft_axis<R, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      k_fft_axis<R, -1><<<blocks, 256, sm, s>>>(data, len, inner, nlines, cb, tw[a]);
    } else {
      CK(cudaFuncSetAttribute(k_fft_axis<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      k_fft_axis<R, 1><<<blocks, 256, sm, s>>>(data, len, inner, nlines, cb, tw[a]);
    }
    CK(cudaGetLastError());
  }
  return SCABEM_OK;
}

// Columns per CTA for the axis-0 stages: 16 (complex64) or 8 (complex128),
// halved until the two ping-pong buffers fit in 192 KB of shared memory.
template <typename R>
int axis0_cb(int P0) {
  int cb = (sizeof(R) == 4) ? 16 : 8;
  while (cb > 1 && 2 * (size_t)P0 * cb * sizeof(cx<R>) > 192 * 1024) cb /= 2;
  return cb;
}

template <typename R>
int fft_conv(scabem_op* op, PrecData<R>& pd, cudaStream_t s) {
  const int n0 = op->n[0], n1 = op->n[1], n2 = op->n[2];
  const int P0 = op->P[0], P1 = op->P[1], P2 = op->P[2];
  const int C = n1 * n2;
  // stage A
  {
    const int cb = axis0_cb<R>(P0);
    const size_t sm = 2 * (size_t)P0 * cb * sizeof(cx<R>);
    CK(cudaFuncSetAttribute(k_axis0<R, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 grid((unsigned)cdiv(C, cb), NFIELD_IN);
    k_axis0<R, -1><<<grid, 512, sm, s>>>(pd.src, pd.stA, n0, P0, P0, C, cb, pd.tw[0]);
    CK(cudaGetLastError());
  }
  prof_mark(op, s);
  // stage B
  {
    const size_t sm = 3 * (size_t)P1 * P2 * sizeof(cx<R>);
    CK(cudaFuncSetAttribute(k_planes<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 grid(P0, NFIELD_IN);
    k_planes<R><<<grid, 512, sm, s>>>(pd.stA, pd.stB, pd.ghat[0], pd.ghat[1], P0, n1, n2, P1, P2, pd.tw[1], pd.tw[2]);
    CK(cudaGetLastError());
  }
  prof_mark(op, s);
  // stage C
  {
    const int cb = axis0_cb<R>(P0);
    const size_t sm = 2 * (size_t)P0 * cb * sizeof(cx<R>);
    CK(cudaFuncSetAttribute(k_axis0<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 grid((unsigned)cdiv(C, cb), NFIELD_OUT);
    k_axis0<R, 1><<<grid, 512, sm, s>>>(pd.stB, pd.grid, P0, n0, P0, C, cb, pd.tw[0]);
    CK(cudaGetLastError());
  }
  return SCABEM_OK;
}

template int make_twiddles<float>(cx<float>*, int, cudaStream_t);
template int make_twiddles<double>(cx<double>*, int, cudaStream_t);
template int fft3d_full<double>(scabem_op*, cx<double>*, const cx<double>* const[3], int, cudaStream_t);
template int fft_conv<float>(scabem_op*, PrecData<float>&, cudaStream_t);
template int fft_conv<double>(scabem_op*, PrecData<double>&, cudaStream_t);
