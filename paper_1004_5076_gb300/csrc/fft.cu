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
//   stage C: inverse FFT along axis 0, keep i0 < n0, written point-major
//            [i0][i1][i2][16] for the interpolation gathers.
// Every FFT is an in-place shared-memory Stockham transform (radix 8, then 4
// or 2) with compile-time power-of-two lengths: each pass loads its
// butterflies into registers, synchronises, and stores them at their sorted
// positions.  One CTA owns whole lines, so each field makes one HBM round trip
// per stage.  The 1/(P0 P1 P2) scale is folded into the stored spectra.
#include <cuda_runtime.h>

#include "common.cuh"

namespace {

constexpr int FFT_THREADS = 512;
constexpr int FFT_LTHREADS = 9;

template <typename R, int DIR>
__device__ __forceinline__ cx<R> rot(cx<R> a) {  // multiply by DIR * j
  return DIR < 0 ? mk(a.im, -a.re) : mk(-a.im, a.re);
}

// complex add / subtract; complex64 as one packed FP32x2 add
__device__ __forceinline__ cx<float> padd(cx<float> a, cx<float> b) {
  const float2 r = __fadd2_rn(make_float2(a.re, a.im), make_float2(b.re, b.im));
  return mk(r.x, r.y);
}
__device__ __forceinline__ cx<float> psub(cx<float> a, cx<float> b) {
  const float2 r = __fadd2_rn(make_float2(a.re, a.im), make_float2(-b.re, -b.im));
  return mk(r.x, r.y);
}
__device__ __forceinline__ cx<double> padd(cx<double> a, cx<double> b) { return a + b; }
__device__ __forceinline__ cx<double> psub(cx<double> a, cx<double> b) { return a - b; }

template <typename R, int DIR>
__device__ __forceinline__ void dft4(cx<R>& a0, cx<R>& a1, cx<R>& a2, cx<R>& a3) {
  cx<R> t0 = padd(a0, a2), t1 = psub(a0, a2), t2 = padd(a1, a3), u = rot<R, DIR>(psub(a1, a3));
  a0 = padd(t0, t2);
  a2 = psub(t0, t2);
  a1 = padd(t1, u);
  a3 = psub(t1, u);
}

template <typename R, int RAD, int DIR>
__device__ __forceinline__ void dft(cx<R>* v) {
  if constexpr (RAD == 2) {
    const cx<R> t = v[0];
    v[0] = t + v[1];
    v[1] = t - v[1];
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
    const cx<R> w1 = s * (o1 + rot<R, DIR>(o1));
    const cx<R> w2 = rot<R, DIR>(o2);
    const cx<R> w3 = s * (rot<R, DIR>(o3) - o3);
    v[0] = padd(e0, o0);
    v[4] = psub(e0, o0);
    v[1] = padd(e1, w1);
    v[5] = psub(e1, w1);
    v[2] = padd(e2, w2);
    v[6] = psub(e2, w2);
    v[3] = padd(e3, w3);
    v[7] = psub(e3, w3);
  }
}

// One in-place Stockham pass of radix 2^LR over the 2^lnl lines of length
// N = 2^LN; element j of line l lives at buf[l*ls + j*es].  2^LNS is the
// product of the radices of the previous passes.  Consecutive threads take
// consecutive lines.  TOTL = log2 of the largest element count a caller
// passes, which bounds the butterflies each thread holds.
template <typename R, int LN, int LR, int LNS, int DIR, int TOTL>
__device__ __forceinline__ void pass_ip(cx<R>* buf, int lnl, int ls, int es, const cx<R>* tw) {
  constexpr int RAD = 1 << LR;
  constexpr int LPER = LN - LR;
  constexpr int NSM = (1 << LNS) - 1;
  constexpr int LTS = LN - LNS - LR;
  constexpr int MB0 = TOTL - LR - FFT_LTHREADS;
  constexpr int MAXB = MB0 > 0 ? (1 << MB0) : 1;
  const int nb = 1 << (lnl + LPER);
  const int lmask = (1 << lnl) - 1;
  cx<R> v[MAXB][RAD];
  int dst[MAXB];
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = threadIdx.x + i * FFT_THREADS;
    if (b < nb) {
      const int line = b & lmask;
      const int j = b >> lnl;
      const cx<R>* s = buf + line * ls;
#pragma unroll
      for (int r = 0; r < RAD; ++r) v[i][r] = s[(j + (r << LPER)) * es];
      if (LNS > 0) {
        const int k = j & NSM;
#pragma unroll
        for (int r = 1; r < RAD; ++r) {
          cx<R> t = tw[(r * k) << LTS];
          if (DIR > 0) t = conj(t);
          v[i][r] = v[i][r] * t;
        }
      }
      dft<R, RAD, DIR>(v[i]);
      dst[i] = line * ls + ((((j >> LNS) << (LNS + LR)) + (j & NSM)) * es);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = threadIdx.x + i * FFT_THREADS;
    if (b < nb) {
#pragma unroll
      for (int r = 0; r < RAD; ++r) buf[dst[i] + ((r << LNS) * es)] = v[i][r];
    }
  }
  __syncthreads();
}

template <typename R, int LN, int LNS, int DIR, int TOTL>
__device__ __forceinline__ void fft_ip(cx<R>* buf, int lnl, int ls, int es, const cx<R>* tw) {
  if constexpr (LNS < LN) {
    constexpr int REM = LN - LNS;
    constexpr int LR = REM >= 3 ? 3 : REM;
    pass_ip<R, LN, LR, LNS, DIR, TOTL>(buf, lnl, ls, es, tw);
    fft_ip<R, LN, LNS + LR, DIR, TOTL>(buf, lnl, ls, es, tw);
  }
}

// FFT of 2^lnl lines of length 2^ln (3 <= ln <= 10), all threads of the CTA.
template <typename R, int DIR, int TOTL>
__device__ __forceinline__ void fft_lines(cx<R>* buf, int ln, int lnl, int ls, int es, const cx<R>* tw) {
  switch (ln) {
    case 3: fft_ip<R, 3, 0, DIR, TOTL>(buf, lnl, ls, es, tw); break;
    case 4: fft_ip<R, 4, 0, DIR, TOTL>(buf, lnl, ls, es, tw); break;
    case 5: fft_ip<R, 5, 0, DIR, TOTL>(buf, lnl, ls, es, tw); break;
    case 6: fft_ip<R, 6, 0, DIR, TOTL>(buf, lnl, ls, es, tw); break;
    case 7: fft_ip<R, 7, 0, DIR, TOTL>(buf, lnl, ls, es, tw); break;
    case 8: fft_ip<R, 8, 0, DIR, TOTL>(buf, lnl, ls, es, tw); break;
    case 9: fft_ip<R, 9, 0, DIR, TOTL>(buf, lnl, ls, es, tw); break;
    default: fft_ip<R, 10, 0, DIR, TOTL>(buf, lnl, ls, es, tw); break;
  }
}

__host__ __device__ inline int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// largest element count (log2) one CTA transforms: complex64 8192, complex128 4096
template <typename R>
struct Tot {
  static constexpr int L = sizeof(R) == 4 ? 13 : 12;
};

// ---------------------------------------------------------------- stage A / C
// Stage A on the active columns acol[0 .. nac) of the [field][i0][c] layout
// (C columns per i0); one CTA owns CB of them for one field over the whole
// axis 0 (smem: [P0][CB], lines = columns).  Inputs i0 >= n_in are zero.
// The output has Cout columns per (field, k0): active column j goes to
// column j (compact, Cout = nac) or to acol[j] (whole planes, Cout = C).
template <typename R>
__global__ void __launch_bounds__(FFT_THREADS) k_axis0(const cx<R>* __restrict__ in, cx<R>* __restrict__ out,
                                                       int n_in, int P0, int C, const int32_t* __restrict__ acol,
                                                       int nac, int CB, const cx<R>* __restrict__ tw,
                                                       int64_t cs_in, int64_t cs_out, int64_t Cout, int compact) {
  extern __shared__ unsigned char smem_raw[];
  cx<R>* tws = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* b0 = tws + P0;
  in += blockIdx.z * cs_in;  // right-hand side blockIdx.z
  out += blockIdx.z * cs_out;
  const int f = blockIdx.y;
  const int a0 = blockIdx.x * CB;
  const int lcb = ilog2(CB);
  for (int i = threadIdx.x; i < P0; i += FFT_THREADS) tws[i] = tw[i];
  const int64_t fin = (int64_t)f * n_in * C;
  for (int idx = threadIdx.x; idx < P0 * CB; idx += FFT_THREADS) {
    const int i0 = idx >> lcb, l = idx & (CB - 1);
    cx<R> v = czero<R>();
    if (i0 < n_in && a0 + l < nac) v = in[fin + (int64_t)i0 * C + acol[a0 + l]];
    b0[idx] = v;
  }
  __syncthreads();
  fft_lines<R, -1, Tot<R>::L>(b0, ilog2(P0), lcb, 1, CB, tws);
  const int64_t fout = (int64_t)f * P0 * Cout;
  for (int idx = threadIdx.x; idx < P0 * CB; idx += FFT_THREADS) {
    const int k0 = idx >> lcb, l = idx & (CB - 1);
    if (a0 + l < nac) out[fout + (int64_t)k0 * Cout + (compact ? a0 + l : acol[a0 + l])] = b0[idx];
  }
}

// Stage C with point-major output, on the active columns acol[0 .. nac)
// only (the potentials are read nowhere else; the input holds Cin columns
// per (field, k0), compact or whole planes as stage A wrote them): one CTA owns NC of them for one group of 4
// output fields over axis 0 (line l = field * NC + column) and writes
// out[(i0 * C + c) * 16 + 4 * grp + f] for i0 < n_out, so the 16 potentials of
// a grid point are contiguous and each group of 4 fills whole 32-byte sectors.
template <typename R>
__global__ void __launch_bounds__(FFT_THREADS) k_axis0_pm(const cx<R>* __restrict__ in, cx<R>* __restrict__ out,
                                                          int n_out, int P0, int C, const int32_t* __restrict__ acol,
                                                          int nac, int NC, const cx<R>* __restrict__ tw,
                                                          int64_t cs_in, int64_t cs_out, int64_t Cin, int compact) {
  extern __shared__ unsigned char smem_raw[];
  cx<R>* tws = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* b0 = tws + P0;
  in += blockIdx.z * cs_in;  // right-hand side blockIdx.z
  out += blockIdx.z * cs_out;
  const int grp = blockIdx.y;
  const int a0 = blockIdx.x * NC;
  const int CB = 4 * NC;
  const int lcb = ilog2(CB), lnc = ilog2(NC);
  for (int i = threadIdx.x; i < P0; i += FFT_THREADS) tws[i] = tw[i];
  for (int idx = threadIdx.x; idx < P0 * CB; idx += FFT_THREADS) {
    const int i0 = idx >> lcb, l = idx & (CB - 1);
    const int fl = l >> lnc, cl = l & (NC - 1);
    cx<R> v = czero<R>();
    if (a0 + cl < nac) v = in[((int64_t)(4 * grp + fl) * P0 + i0) * Cin + (compact ? a0 + cl : acol[a0 + cl])];
    b0[idx] = v;
  }
  __syncthreads();
  fft_lines<R, 1, Tot<R>::L>(b0, ilog2(P0), lcb, 1, CB, tws);
  for (int idx = threadIdx.x; idx < n_out * CB; idx += FFT_THREADS) {
    const int k0 = idx >> lcb, l = idx & (CB - 1);
    const int cl = l >> 2, fl = l & 3;  // field fastest: consecutive threads fill a sector
    if (a0 + cl < nac)
      out[((int64_t)k0 * C + acol[a0 + cl]) * NFIELD_OUT + 4 * grp + fl] = b0[(k0 << lcb) + fl * NC + cl];
  }
}

// ---------------------------------------------------------------- warp-owned lines
// FFT of one line of length 2^LN owned by T = 2^(LN-3) consecutive lanes of a
// warp (lane tl of the group).  The first pass reads element j through
// ld(j), the last pass writes element j through st(j, v); the passes in
// between exchange through the line's shared-memory storage line[j*es]
// with warp-level synchronisation only.
template <typename R, int LN, int LNS, int DIR, class LD, class ST>
__device__ __forceinline__ void wline_fft(cx<R>* line, int es, int tl, bool act, const cx<R>* tw, const LD& ld,
                                          const ST& st) {
  if constexpr (LNS < LN) {
    constexpr int REM = LN - LNS;
    constexpr int LR = REM >= 3 ? 3 : REM;
    constexpr int RAD = 1 << LR;
    constexpr int LT = LN - 3;
    constexpr int LPER = LN - LR;
    constexpr int NBT = 1 << (LPER - LT);  // butterflies per lane
    constexpr int NSM = (1 << LNS) - 1;
    constexpr int LTS = LN - LNS - LR;
    constexpr bool FIRST = LNS == 0, LAST = LNS + LR == LN;
    cx<R> v[NBT][RAD];
    int dst[NBT];
    if (act) {
#pragma unroll
      for (int i = 0; i < NBT; ++i) {
        const int j = tl + (i << LT);
#pragma unroll
        for (int r = 0; r < RAD; ++r) {
          const int e = j + (r << LPER);
          v[i][r] = FIRST ? ld(e) : line[e * es];
        }
        if (LNS > 0) {
          const int k = j & NSM;
#pragma unroll
          for (int r = 1; r < RAD; ++r) {
            cx<R> t = tw[(r * k) << LTS];
            if (DIR > 0) t = conj(t);
            v[i][r] = v[i][r] * t;
          }
        }
        dft<R, RAD, DIR>(v[i]);
        dst[i] = ((j >> LNS) << (LNS + LR)) + (j & NSM);
      }
    }
    if (!LAST) __syncwarp();
    if (act) {
#pragma unroll
      for (int i = 0; i < NBT; ++i)
#pragma unroll
        for (int r = 0; r < RAD; ++r) {
          const int e = dst[i] + (r << LNS);
          if (LAST)
            st(e, v[i][r]);
          else
            line[e * es] = v[i][r];
        }
    }
    if (!LAST) {
      __syncwarp();
      wline_fft<R, LN, LNS + LR, DIR>(line, es, tl, act, tw, ld, st);
    }
  }
}

// Runs f(l, line, tl, act) for lines l < nlines spread over the warps of the
// CTA (2^(5-LT) lines per warp); trip counts are uniform within a warp.
template <int LN, class F>
__device__ __forceinline__ void for_warp_lines(int nlines, const F& f) {
  constexpr int LT = LN - 3;
  constexpr int LPW = 32 >> LT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int tl = lane & ((1 << LT) - 1), sub = lane >> LT;
  for (int l0 = warp * LPW; l0 < nlines; l0 += nw * LPW) {
    const int l = l0 + sub;
    f(l < nlines ? l : 0, tl, l < nlines);
  }
}

// ---------------------------------------------------------------- stage B
// One CTA per (k0 plane, source field).  Source fields:
//   0..3  exterior J (x, y, z, div)  -> outputs 0..3 with G_e
//   4..7  interior J                 -> outputs 8..11 with G_i
//   8..11 exterior M                 -> outputs 4..7 with G_e and 12..15 with -G_i
// The plane lives in shared memory with row stride P2 + 2; S holds the
// forward spectrum, W the working plane of one output.  The forward row pass
// reads the physical n1 x n2 corner straight from global memory, the forward
// column pass skips the zero rows, the Green multiply is applied as the
// inverse column pass loads S, only the n1 physical rows are kept, and the
// inverse row pass writes the physical corner straight to global memory.
constexpr int PLANE_THREADS = 256;

template <typename R, int L1, int L2>
__global__ void __launch_bounds__(PLANE_THREADS) k_planes(const cx<R>* __restrict__ A, cx<R>* __restrict__ B,
                                                          const cx<R>* __restrict__ ghE,
                                                          const cx<R>* __restrict__ ghI, int P0, int n1, int n2,
                                                          const cx<R>* __restrict__ tw1,
                                                          const cx<R>* __restrict__ tw2, int ident, int64_t cs) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int P1 = 1 << L1, P2 = 1 << L2;
  A += blockIdx.z * cs;  // right-hand side blockIdx.z
  B += blockIdx.z * cs;
  constexpr int LS = P2 + 2;
  constexpr int plane = P1 * LS;
  cx<R>* t1 = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* t2 = t1 + P1;
  cx<R>* S = t2 + P2;
  cx<R>* W = S + plane;
  const int k0 = blockIdx.x;
  const int f = blockIdx.y;
  for (int i = threadIdx.x; i < P1; i += PLANE_THREADS) t1[i] = tw1[i];
  for (int i = threadIdx.x; i < P2; i += PLANE_THREADS) t2[i] = tw2[i];
  __syncthreads();
  const int64_t C = (int64_t)n1 * n2;
  const cx<R>* src = A + ((int64_t)f * P0 + k0) * C;
  // forward rows (axis 2): the n1 non-zero rows, read from global memory
  for_warp_lines<L2>(n1, [&](int i1, int tl, bool act) {
    cx<R>* row = S + i1 * LS;
    wline_fft<R, L2, 0, -1>(
        row, 1, tl, act, t2, [&](int e) { return e < n2 ? src[i1 * n2 + e] : czero<R>(); },
        [&](int e, cx<R> v) { row[e] = v; });
  });
  __syncthreads();
  // forward columns (axis 1): rows >= n1 are zero and are not read
  for_warp_lines<L1>(P2, [&](int k2, int tl, bool act) {
    cx<R>* col = S + k2;
    wline_fft<R, L1, 0, -1>(
        col, LS, tl, act, t1, [&](int e) { return e < n1 ? col[e * LS] : czero<R>(); },
        [&](int e, cx<R> v) { col[e * LS] = v; });
  });
  __syncthreads();

  const int h1 = P1 / 2 + 1, h2 = P2 / 2 + 1;
  const int q0 = min(k0, P0 - k0);
  const int nout = (!ident && f >= 8) ? 2 : 1;
  for (int which = 0; which < nout; ++which) {
    int fo;
    const cx<R>* gh;
    R sgn = R(1);
    if (ident) {  // transposed apply: each of the 16 fields with its medium's function
      fo = f;
      gh = f < 8 ? ghE : ghI;
    } else if (f < 4) {
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
    // inverse columns: load S times the Green spectrum, keep rows < n1 in W
    for_warp_lines<L1>(P2, [&](int k2, int tl, bool act) {
      const cx<R>* scol = S + k2;
      cx<R>* wcol = W + k2;
      const cx<R>* gcol = g0 + min(k2, P2 - k2) * h1;
      wline_fft<R, L1, 0, 1>(
          wcol, LS, tl, act, t1,
          [&](int e) { return sgn * (scol[e * LS] * gcol[min(e, P1 - e)]); },
          [&](int e, cx<R> v) {
            if (e < n1) wcol[e * LS] = v;
          });
    });
    __syncthreads();
    // inverse rows: the n1 physical rows, written straight to global memory
    cx<R>* dst = B + ((int64_t)fo * P0 + k0) * C;
    for_warp_lines<L2>(n1, [&](int i1, int tl, bool act) {
      cx<R>* row = W + i1 * LS;
      wline_fft<R, L2, 0, 1>(
          row, 1, tl, act, t2, [&](int e) { return row[e]; },
          [&](int e, cx<R> v) {
            if (e < n2) dst[i1 * n2 + e] = v;
          });
    });
    __syncthreads();
  }
}

template <typename R>
using PlanesFn = void (*)(const cx<R>*, cx<R>*, const cx<R>*, const cx<R>*, int, int, int, const cx<R>*,
                          const cx<R>*, int, int64_t);

template <typename R, int L1, int L2>
PlanesFn<R> planes_fn() {
  if constexpr (L1 + L2 <= 12) return k_planes<R, L1, L2>;
  else return nullptr;
}

template <typename R, int L1>
PlanesFn<R> planes_row(int l2) {
  switch (l2) {
    case 3: return planes_fn<R, L1, 3>();
    case 4: return planes_fn<R, L1, 4>();
    case 5: return planes_fn<R, L1, 5>();
    case 6: return planes_fn<R, L1, 6>();
    case 7: return planes_fn<R, L1, 7>();
    default: return nullptr;
  }
}

// ---------------------------------------------------------------- stage B, 64 x 64 planes
// The same plane step specialised to P1 = P2 = 64 (n1 = n2 = 32), the usual
// cross-section of a guide grid.  A 64-point line belongs to eight lanes:
// lane t holds elements t + 8r, transforms over r (radix 8), multiplies by
// w64^(t k) and swaps through a per-line scratch so that lane k then holds
// index k of every t; a second radix-8 transform leaves elements k + 8m in
// lane k.  That is the layout the inverse transform starts from, so the
// forward column transform, the Green multiply of each output and the
// inverse column transform run back to back in registers.  Half-zero inputs
// and half-kept outputs use pruned radix-8 transforms.
//
// Shared memory (8-byte words, 16 banks of 8 bytes per half-warp): a plane
// holds rows 0..31 with row i, column k at i*64 + (k ^ g(i)), g(i) =
// 2(i mod 8) ^ 8(i mod 2); row accesses (two rows per half-warp) and column
// accesses (eight rows of two columns per half-warp) are then free of bank
// conflicts.  The per-line scratch puts element (t, k) at 8t + (k + t) mod 8,
// 72 words per line, for the same reason.
constexpr int P64_THREADS = 256;  // 8 warps x 4 lines of 8 lanes: one pass over 32 rows
constexpr int P64_SCR = 72;

__device__ __forceinline__ int swz64(int i, int k) { return i * 64 + (k ^ ((2 * (i & 7)) ^ ((i & 1) << 3))); }

// radix-8 transform of v[0..3] with v[4..7] = 0
template <typename R, int DIR>
__device__ __forceinline__ void dft8_hin(cx<R>* v) {
  const R s = R(0.70710678118654752440);
  cx<R> e0 = v[0], e1 = v[1], e2 = v[2], e3 = v[3];
  cx<R> o0 = v[0], o1 = s * (v[1] + rot<R, DIR>(v[1])), o2 = rot<R, DIR>(v[2]), o3 = s * (rot<R, DIR>(v[3]) - v[3]);
  dft4<R, DIR>(e0, e1, e2, e3);
  dft4<R, DIR>(o0, o1, o2, o3);
  v[0] = e0;
  v[2] = e1;
  v[4] = e2;
  v[6] = e3;
  v[1] = o0;
  v[3] = o1;
  v[5] = o2;
  v[7] = o3;
}

// radix-8 transform keeping outputs 0..3
template <typename R, int DIR>
__device__ __forceinline__ void dft8_hout(cx<R>* v) {
  cx<R> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  cx<R> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<R, DIR>(e0, e1, e2, e3);
  dft4<R, DIR>(o0, o1, o2, o3);
  const R s = R(0.70710678118654752440);
  v[0] = padd(e0, o0);
  v[1] = padd(e1, s * (o1 + rot<R, DIR>(o1)));
  v[2] = padd(e2, rot<R, DIR>(o2));
  v[3] = padd(e3, s * (rot<R, DIR>(o3) - o3));
}

// 64-point transform of one line over its eight lanes (lane t, v[r] =
// element t + 8r on entry, element t + 8m in v[m] on exit); w[k] = w64^(t k).
template <typename R, int DIR, bool HALF_IN, bool HALF_OUT>
__device__ __forceinline__ void line64(cx<R>* v, const cx<R>* w, cx<R>* scr, int t) {
  if (HALF_IN)
    dft8_hin<R, DIR>(v);
  else
    dft<R, 8, DIR>(v);
#pragma unroll
  for (int k = 1; k < 8; ++k) v[k] = v[k] * (DIR < 0 ? w[k] : conj(w[k]));
#pragma unroll
  for (int k = 0; k < 8; ++k) scr[t * 8 + ((k + t) & 7)] = v[k];
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = scr[i * 8 + ((t + i) & 7)];
  __syncwarp();
  if (HALF_OUT)
    dft8_hout<R, DIR>(v);
  else
    dft<R, 8, DIR>(v);
}

template <typename R>
__global__ void __launch_bounds__(P64_THREADS, sizeof(R) == 4 ? 3 : 1)
    k_planes64(const cx<R>* __restrict__ A, cx<R>* __restrict__ B, const cx<R>* __restrict__ ghE,
               const cx<R>* __restrict__ ghI, int P0, const cx<R>* __restrict__ tw64, uint64_t rowmask, int ident,
               int64_t cs) {
  constexpr int NP = 32, H = 33;
  A += blockIdx.z * cs;  // right-hand side blockIdx.z
  B += blockIdx.z * cs;
  extern __shared__ unsigned char smem_raw[];
  cx<R>* W0 = reinterpret_cast<cx<R>*>(smem_raw);  // forward rows, then output 0
  cx<R>* W1 = W0 + NP * 64;                        // output 1
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = lane & 7, sub = lane >> 3;
  cx<R>* scr = W1 + NP * 64 + (warp * 4 + sub) * P64_SCR;
  cx<R> w[8];
  w[0] = mk(R(1), R(0));
#pragma unroll
  for (int k = 1; k < 8; ++k) w[k] = tw64[t * k];
  const int k0 = blockIdx.x, f = blockIdx.y;
  const int i1 = warp * 4 + sub;  // the row this lane works on in the row passes
  // rows no stencil covers are zero in and unused out; the test is per warp
  // (its four rows) so that the line transforms' warp barriers see all lanes
  const bool row_on = ((rowmask >> (warp * 4)) & 0xF) != 0;
  {
    // forward rows: the 32 physical rows, elements >= 32 are zero
    cx<R> v[8];
    if (row_on) {
      const cx<R>* src = A + ((int64_t)f * P0 + k0) * (NP * NP) + i1 * NP;
#pragma unroll
      for (int r = 0; r < 4; ++r) v[r] = src[t + 8 * r];
      line64<R, -1, true, false>(v, w, scr, t);
    } else {
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = czero<R>();
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) W0[swz64(i1, t + 8 * m)] = v[m];
  }
  __syncthreads();

  // source field -> output fields, media and signs (as in k_planes)
  // transposed apply (ident): each of the 16 fields with its medium's function
  const int nout = (!ident && f >= 8) ? 2 : 1;
  const int q0 = min(k0, P0 - k0);
  const cx<R>* ga = ident ? (f < 8 ? ghE : ghI) : ((f >= 4 && f < 8) ? ghI : ghE);  // output 0
  const int foa = ident ? f : (f < 4 ? f : (f < 8 ? 8 + (f - 4) : 4 + (f - 8)));
  const int fob = 12 + (f - 8);  // output 1 (f >= 8), interior medium, sign -1
  ga += (int64_t)q0 * H * H;
  const cx<R>* gb = ghI + (int64_t)q0 * H * H;

  // columns: forward transform (rows >= 32 zero), Green multiply, inverse
  // transform, rows < 32 kept in W0 / W1 (a column is read and rewritten by
  // the same eight lanes)
#pragma unroll 1
  for (int it = 0; it < 2; ++it) {
    const int c = it * 32 + warp * 4 + sub;
    cx<R> x[8];
#pragma unroll
    for (int r = 0; r < 4; ++r) x[r] = W0[swz64(t + 8 * r, c)];
    line64<R, -1, true, false>(x, w, scr, t);
    const int cg = min(c, 64 - c) * H;
#pragma unroll 1
    for (int o = 0; o < nout; ++o) {
      const cx<R>* gp = (o ? gb : ga) + cg;
      cx<R> v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int e = t + 8 * m;
        v[m] = x[m] * gp[min(e, 64 - e)];
        if (o) v[m] = -v[m];
      }
      line64<R, 1, false, true>(v, w, scr, t);
      cx<R>* Wo = o ? W1 : W0;
#pragma unroll
      for (int m = 0; m < 4; ++m) Wo[swz64(t + 8 * m, c)] = v[m];
    }
  }
  __syncthreads();

  // inverse rows, the 32 physical columns written to global memory
#pragma unroll 1
  for (int o = 0; o < nout && row_on; ++o) {
    const cx<R>* Wo = o ? W1 : W0;
    cx<R> v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = Wo[swz64(i1, t + 8 * r)];
    line64<R, 1, false, true>(v, w, scr, t);
    cx<R>* dst = B + ((int64_t)(o ? fob : foa) * P0 + k0) * (NP * NP) + i1 * NP;
#pragma unroll
    for (int m = 0; m < 4; ++m) dst[t + 8 * m] = v[m];
  }
}

// ---------------------------------------------------------------- stage B, direct
// (In the transposed apply, ident = 1, medium m takes fields 8m .. 8m+7 to
// the same fields, no sign.)
// Stage B as a direct sum over the active (i1, i2) columns: per (k0 plane,
// medium) the 8 source fields of that medium (its J set and the M set) are
// convolved with gt[q0][|d1|][|d2|] (the axis-0 transform of the spatial
// Green table):  out_v(i) = sum over active j of gt(|i1 - j1|, |i2 - j2|)
// src_v(j).  This is the linear convolution that the zero-padded 2-D FFTs
// compute (offsets never reach the padding), evaluated only on the columns
// that are read.  Medium 0: J_e (0..3), M (8..11) -> outputs 0..3, 4..7;
// medium 1: J_i (4..7), M (8..11) -> outputs 8..11 and -(12..15).  One
// thread per output column, 8 accumulators; each table value serves the 8
// fields, and the source values are shared-memory broadcasts.
constexpr int PD_THREADS = 128;

// acc[v] += t * s[v], v < 8; complex64 keeps P + j Q parts (packed FP32x2)
template <typename R>
struct Acc8;
template <>
struct Acc8<float> {
  float2 P[8], Q[8];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int v = 0; v < 8; ++v) P[v] = Q[v] = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ void mac(cx<float> t, const cx<float>* s) {
    const float2 tr = make_float2(t.re, t.re), ti = make_float2(t.im, t.im);
    const float4* s4 = reinterpret_cast<const float4*>(s);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4 w = s4[u];
      const float2 a = make_float2(w.x, w.y), b = make_float2(w.z, w.w);
      P[2 * u] = __ffma2_rn(tr, a, P[2 * u]);
      Q[2 * u] = __ffma2_rn(ti, a, Q[2 * u]);
      P[2 * u + 1] = __ffma2_rn(tr, b, P[2 * u + 1]);
      Q[2 * u + 1] = __ffma2_rn(ti, b, Q[2 * u + 1]);
    }
  }
  __device__ __forceinline__ cx<float> get(int v) const { return mk(P[v].x - Q[v].y, P[v].y + Q[v].x); }
};
template <>
struct Acc8<double> {
  cx<double> a[8];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int v = 0; v < 8; ++v) a[v] = czero<double>();
  }
  __device__ __forceinline__ void mac(cx<double> t, const cx<double>* s) {
#pragma unroll
    for (int v = 0; v < 8; ++v) cfma(a[v], t, s[v]);
  }
  __device__ __forceinline__ cx<double> get(int v) const { return a[v]; }
};

template <typename R>
__global__ void __launch_bounds__(PD_THREADS) k_planes_direct(const cx<R>* __restrict__ A, cx<R>* __restrict__ B,
                                                              const cx<R>* __restrict__ gtE,
                                                              const cx<R>* __restrict__ gtI, int P0, int C,
                                                              const int32_t* __restrict__ acol,
                                                              const int32_t* __restrict__ acoord, int nac, int R1,
                                                              int R2, int ident, int64_t cs, int compact) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  A += blockIdx.z * cs;  // right-hand side blockIdx.z
  B += blockIdx.z * cs;
  cx<R>* src = reinterpret_cast<cx<R>*>(smem_raw);  // [nac][8]
  cx<R>* T = src + (int64_t)nac * 8;                 // [R1][R2]
  int32_t* crd = reinterpret_cast<int32_t*>(T + R1 * R2);
  const int k0 = blockIdx.x, med = blockIdx.y;
  const int q0 = min(k0, P0 - k0);
  const cx<R>* gt = (med ? gtI : gtE) + (int64_t)q0 * R1 * R2;
  for (int i = threadIdx.x; i < R1 * R2; i += PD_THREADS) T[i] = gt[i];
  for (int idx = threadIdx.x; idx < nac * 8; idx += PD_THREADS) {
    const int v = idx / nac, j = idx - v * nac;  // consecutive threads: consecutive columns of one field
    const int f = ident ? 8 * med + v : (v < 4 ? (med ? 4 + v : v) : 8 + (v - 4));
    src[j * 8 + v] = A[((int64_t)f * P0 + k0) * C + (compact ? j : acol[j])];
  }
  for (int i = threadIdx.x; i < nac; i += PD_THREADS) crd[i] = acoord[i];
  __syncthreads();
  for (int i = threadIdx.x; i < nac; i += PD_THREADS) {
    const int ci = crd[i];
    const int i1 = ci >> 16, i2 = ci & 0xffff;
    Acc8<R> acc;
    acc.zero();
    for (int j = 0; j < nac; ++j) {
      const int cj = crd[j];
      const int d1 = abs(i1 - (cj >> 16)), d2 = abs(i2 - (cj & 0xffff));
      acc.mac(T[d1 * R2 + d2], src + j * 8);
    }
    const int64_t c = compact ? i : acol[i];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int fo = ident ? 8 * med + v : (med ? (v < 4 ? 8 + v : 12 + (v - 4)) : v);
      const cx<R> val = acc.get(v);
      B[((int64_t)fo * P0 + k0) * C + c] = (!ident && med && v >= 4) ? -val : val;
    }
  }
}

// Compiled plane sizes: (2^l1) x (2^l2) with 3 <= l1, l2 <= 7 and l1 + l2 <= 12.
template <typename R>
PlanesFn<R> planes_kernel(int l1, int l2) {
  switch (l1) {
    case 3: return planes_row<R, 3>(l2);
    case 4: return planes_row<R, 4>(l2);
    case 5: return planes_row<R, 5>(l2);
    case 6: return planes_row<R, 6>(l2);
    case 7: return planes_row<R, 7>(l2);
    default: return nullptr;
  }
}

// ---------------------------------------------------------------- generic 3-D FFT (set-up, complex128)
template <typename R, int DIR>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_axis(cx<R>* data, int len, int inner, int64_t nlines, int CB,
                                                          const cx<R>* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  cx<R>* tws = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* b0 = tws + len;
  const int64_t L0 = (int64_t)blockIdx.x * CB;
  const int lcb = ilog2(CB);
  for (int i = threadIdx.x; i < len; i += FFT_THREADS) tws[i] = tw[i];
  for (int idx = threadIdx.x; idx < len * CB; idx += FFT_THREADS) {
    const int j = idx >> lcb, l = idx & (CB - 1);
    const int64_t L = L0 + l;
    cx<R> v = czero<R>();
    if (L < nlines) v = data[(L / inner) * ((int64_t)len * inner) + (L % inner) + (int64_t)j * inner];
    b0[idx] = v;
  }
  __syncthreads();
  fft_lines<R, DIR, Tot<R>::L>(b0, ilog2(len), lcb, 1, CB, tws);
  for (int idx = threadIdx.x; idx < len * CB; idx += FFT_THREADS) {
    const int j = idx >> lcb, l = idx & (CB - 1);
    const int64_t L = L0 + l;
    if (L < nlines) data[(L / inner) * ((int64_t)len * inner) + (L % inner) + (int64_t)j * inner] = b0[idx];
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

// Lines per CTA for a transform of length len: up to 2^Tot<R>::L elements,
// at most 16 lines.
template <typename R>
int lines_per_cta(int len) {
  int cb = (1 << Tot<R>::L) / len;
  if (cb > 16) cb = 16;
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

// Full-length transform along one axis of a P0 x P1 x P2 array (set-up).
template <typename R>
int fft_axis_full(scabem_op* op, cx<R>* data, int a, const cx<R>* tw, int dir, cudaStream_t s) {
  const int64_t total = (int64_t)op->P[0] * op->P[1] * op->P[2];
  const int len = op->P[a];
  int inner = 1;
  for (int b = a + 1; b < 3; ++b) inner *= op->P[b];
  const int64_t nlines = total / len;
  const int cb = lines_per_cta<R>(len);
  const size_t sm = (size_t)len * (cb + 1) * sizeof(cx<R>);
  const int blocks = (int)cdiv(nlines, cb);
  if (dir < 0) {
    CK(cudaFuncSetAttribute(k_fft_axis<R, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_fft_axis<R, -1><<<blocks, FFT_THREADS, sm, s>>>(data, len, inner, nlines, cb, tw);
  } else {
    CK(cudaFuncSetAttribute(k_fft_axis<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_fft_axis<R, 1><<<blocks, FFT_THREADS, sm, s>>>(data, len, inner, nlines, cb, tw);
  }
  CK(cudaGetLastError());
  return SCABEM_OK;
}

template <typename R>
int fft3d_full(scabem_op* op, cx<R>* data, const cx<R>* const tw[3], int dir, cudaStream_t s) {
  for (int a = 0; a < 3; ++a) {
    int rc = fft_axis_full<R>(op, data, a, tw[a], dir, s);
    if (rc) return rc;
  }
  return SCABEM_OK;
}

// Lines per CTA of the pruned axis-0 stages: at most 8, so that the few
// active columns still spread over the SMs.
template <typename R>
int pruned_lines(int P0) {
  const int l = lines_per_cta<R>(P0);
  return l < 8 ? l : 8;
}

// stage C: 16 fields [field][k0][c] -> point-major grid [i0][c][16], active columns
template <typename R>
static int axis0_inverse(scabem_op* op, PrecData<R>& pd, cudaStream_t s, int ncol) {
  const int n0 = op->n[0], P0 = op->P[0];
  const int C = op->n[1] * op->n[2];
  const int lines = op->a0_lines > 0 ? op->a0_lines : pruned_lines<R>(P0);
  const int nc = lines >= 4 ? lines / 4 : 1;  // P0 <= 1024: 4 lines fit
  const size_t sm = (size_t)P0 * (4 * nc + 1) * sizeof(cx<R>);
  if (int rc_ = set_max_smem(op->device, (const void*)k_axis0_pm<R>, (int)sm)) return rc_;
  k_axis0_pm<R><<<dim3((unsigned)cdiv(op->nac, nc), NFIELD_OUT / 4, ncol), FFT_THREADS, sm, s>>>(
      pd.stB, pd.grid, n0, P0, C, op->acol, (int)op->nac, nc, pd.tw[0], col_stride_st(op), col_stride_grid(op),
      op->cst, op->tdirect ? 1 : 0);
  CK(cudaGetLastError());
  return SCABEM_OK;
}

template <typename R>
int fft_conv(scabem_op* op, PrecData<R>& pd, cudaStream_t s, bool adjoint, int ncol) {
  const int n0 = op->n[0], n1 = op->n[1], n2 = op->n[2];
  const int nf = adjoint ? NFIELD_OUT : NFIELD_IN;  // fields transformed along axis 0
  const int id = adjoint ? 1 : 0;
  const int P0 = op->P[0], P1 = op->P[1], P2 = op->P[2];
  const int C = n1 * n2;
  if (op->nac == 0) {
    set_error("grid: no grid point is covered by a stencil");
    return SCABEM_E_ARG;
  }
  const int cb = op->a0_lines > 0 ? op->a0_lines : pruned_lines<R>(P0);
  const size_t sm0 = (size_t)P0 * (cb + 1) * sizeof(cx<R>);
  // stage A
  if (int rc_ = set_max_smem(op->device, (const void*)k_axis0<R>, (int)sm0)) return rc_;
  k_axis0<R><<<dim3((unsigned)cdiv(op->nac, cb), nf, ncol), FFT_THREADS, sm0, s>>>(
      pd.src, pd.stA, n0, P0, C, op->acol, (int)op->nac, cb, pd.tw[0], col_stride_grid(op), col_stride_st(op),
      op->cst, op->tdirect ? 1 : 0);
  CK(cudaGetLastError());
  prof_mark(op, s);
  // stage B
  if (op->tdirect) {
    const size_t sm = ((size_t)op->nac * 8 + (size_t)op->R1 * op->R2) * sizeof(cx<R>) + sizeof(int32_t) * op->nac;
    if (int rc_ = set_max_smem(op->device, (const void*)k_planes_direct<R>, (int)sm)) return rc_;
    k_planes_direct<R><<<dim3(P0, 2, ncol), PD_THREADS, sm, s>>>(pd.stA, pd.stB, pd.gt[0], pd.gt[1], P0,
                                                                 (int)op->cst, op->acol, op->acoord, (int)op->nac,
                                                                 op->R1, op->R2, id, col_stride_st(op), 1);
    CK(cudaGetLastError());
    prof_mark(op, s);
    return axis0_inverse(op, pd, s, ncol);
  }
  if (P1 == 64 && P2 == 64) {
    const size_t sm = ((size_t)2 * 32 * 64 + (size_t)(P64_THREADS / 8) * P64_SCR) * sizeof(cx<R>);
    if (int rc_ = set_max_smem(op->device, (const void*)k_planes64<R>, (int)sm)) return rc_;
    k_planes64<R><<<dim3(P0, nf, ncol), P64_THREADS, sm, s>>>(pd.stA, pd.stB, pd.ghat[0], pd.ghat[1], P0, pd.tw[1],
                                                              op->rowmask, id, col_stride_st(op));
    CK(cudaGetLastError());
    prof_mark(op, s);
    return axis0_inverse(op, pd, s, ncol);
  }
  const size_t sm1 = ((size_t)P1 + P2 + 2 * (size_t)P1 * (P2 + 2)) * sizeof(cx<R>);
  PlanesFn<R> fn = planes_kernel<R>(ilog2(P1), ilog2(P2));
  if (!fn) {
    set_error("grid: the y and z transform sizes must be in [8, 128]");
    return SCABEM_E_ARG;
  }
  if (int rc_ = set_max_smem(op->device, (const void*)fn, (int)sm1)) return rc_;
  fn<<<dim3(P0, nf, ncol), PLANE_THREADS, sm1, s>>>(pd.stA, pd.stB, pd.ghat[0], pd.ghat[1], P0, n1, n2, pd.tw[1],
                                                  pd.tw[2], id, col_stride_st(op));
  CK(cudaGetLastError());
  prof_mark(op, s);
  return axis0_inverse(op, pd, s, ncol);
}

template int make_twiddles<float>(cx<float>*, int, cudaStream_t);
template int make_twiddles<double>(cx<double>*, int, cudaStream_t);
template int fft3d_full<double>(scabem_op*, cx<double>*, const cx<double>* const[3], int, cudaStream_t);
template int fft_axis_full<double>(scabem_op*, cx<double>*, int, const cx<double>*, int, cudaStream_t);
template int fft_conv<float>(scabem_op*, PrecData<float>&, cudaStream_t, bool, int);
template int fft_conv<double>(scabem_op*, PrecData<double>&, cudaStream_t, bool, int);
