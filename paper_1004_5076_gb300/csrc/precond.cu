// Circulant preconditioner for the plain-surface block A_LL of a straight
// extruded guide (Appendix B: on a mesh that repeats along the guide, A_LL
// over the regular slices is block Toeplitz; a block circulant close to it
// is inverted with FFTs over the slice index; the absorber rows keep the
// block-diagonal preconditioner).
//
// Set-up: the regular slices' plain-surface edges are put in one local
// order (translates of the first slice, with the orientation sign of each
// edge); the operator's own columns give the blocks T[d] = A(slice j + d,
// slice j) (the grid operator is translation invariant up to the grid).
// Strang's circulant keeps c_k = T[k] for k <= R/2 and T[k - R] above, from
// the columns of the middle slice; T. Chan's optimal circulant averages each
// wrapped diagonal, c_k = ((R - k) T[k] + k T[k - R]) / R, from the columns
// of the first and the last slice.  The DFT blocks
// C_f = sum_k c_k exp(-2 pi i f k / R) are inverted one per CTA by
// Gauss-Jordan elimination with partial pivoting.
// Apply: v (periodic unknowns, signed) -> DFT over the slices -> C_f^-1 per
// frequency -> inverse DFT -> z, after the block-diagonal preconditioner has
// written every unknown.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"

using cd = cx<double>;

namespace {

constexpr int CIRC_THREADS = 256;

__device__ __forceinline__ cd twiddle(const cd* tw, int64_t e, int R) {
  return tw[(int)(((e % R) + R) % R)];  // exp(-2 pi i e / R)
}

// c[k][i][j] += w_k T[d_k] for the batch of columns j0 .. j0 + kb - 1 of the
// source slice: Y holds A applied to sgn[src][j] e_idx[src][j] (column
// j - j0, leading dimension N), and the block of offset d is read from the
// rows of slice src + d.  mode 0 (Strang, source = the middle slice R/2):
// d = k for k <= R/2, k - R above, weight 1 (0 when slice src + d does not
// exist); mode 1 (Chan, source = slice 0): d = k, weight (R - k) / R;
// mode 2 (Chan, source = slice R - 1): d = k - R, weight k / R.
template <typename R_>
__global__ void k_circ_gather(const cx<R_>* __restrict__ Y, int64_t N, int kb, int j0, const int32_t* __restrict__ idx,
                              const double* __restrict__ sgn, int R, int m, int src, int mode, cd* __restrict__ c) {
  const int64_t tot = (int64_t)R * m * kb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int jj = (int)(t % kb);
    const int i = (int)((t / kb) % m);
    const int k = (int)(t / ((int64_t)kb * m));
    const int d = mode == 0 ? (k <= R / 2 ? k : k - R) : (mode == 1 ? k : k - R);
    const double w = mode == 0 ? 1.0 : (mode == 1 ? (double)(R - k) / R : (double)k / R);
    const int row = src + d;
    if (row >= 0 && row < R && w != 0.0) {
      const cx<R_> y = Y[(int64_t)jj * N + idx[row * m + i]];
      const double sw = w * sgn[row * m + i];
      c[((int64_t)k * m + i) * m + j0 + jj] += mk(sw * (double)y.re, sw * (double)y.im);
    }
  }
}

// C_f[i][j] = sum_k c_k[i][j] exp(-2 pi i f k / R): grid R, threads over (i, j)
__global__ void k_circ_dft_blocks(const cd* __restrict__ c, const cd* __restrict__ tw, int R, int m,
                                  cd* __restrict__ C) {
  const int f = blockIdx.x;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    cd acc = mk(0.0, 0.0);
    for (int k = 0; k < R; ++k) acc += c[(int64_t)k * m * m + e] * twiddle(tw, (int64_t)f * k, R);
    C[(int64_t)f * m * m + e] = acc;
  }
}

// Inverse of the m x m block C_f (one CTA per f) by Gauss-Jordan elimination
// with partial pivoting, in place in a (destroyed) and b (the inverse).
// A zero pivot sets *bad.
__global__ void __launch_bounds__(CIRC_THREADS) k_circ_invert(cd* __restrict__ A, cd* __restrict__ B, int m,
                                                            int* __restrict__ bad) {
  extern __shared__ unsigned char smem_raw[];
  cd* fac = reinterpret_cast<cd*>(smem_raw);  // m column factors
  __shared__ double bv[CIRC_THREADS];
  __shared__ int bi[CIRC_THREADS];
  cd* a = A + (int64_t)blockIdx.x * m * m;
  cd* b = B + (int64_t)blockIdx.x * m * m;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) b[e] = mk(e / m == e % m ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int col = 0; col < m; ++col) {
    // pivot: the largest |a[r][col]|, r >= col
    double best = -1.0;
    int arg = col;
    for (int r = col + threadIdx.x; r < m; r += blockDim.x) {
      const cd v = a[(int64_t)r * m + col];
      const double mag = v.re * v.re + v.im * v.im;
      if (mag > best) {
        best = mag;
        arg = r;
      }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = arg;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st && (bv[threadIdx.x + st] > bv[threadIdx.x] ||
                               (bv[threadIdx.x + st] == bv[threadIdx.x] && bi[threadIdx.x + st] < bi[threadIdx.x]))) {
        bv[threadIdx.x] = bv[threadIdx.x + st];
        bi[threadIdx.x] = bi[threadIdx.x + st];
      }
      __syncthreads();
    }
    const int piv = bi[0];
    if (!(bv[0] > 0.0)) {
      if (threadIdx.x == 0) atomicOr(bad, 1);
      return;  // the whole CTA leaves together (bv[0] is shared)
    }
    // swap rows col and piv
    if (piv != col)
      for (int e = threadIdx.x; e < m; e += blockDim.x) {
        cd t = a[(int64_t)col * m + e];
        a[(int64_t)col * m + e] = a[(int64_t)piv * m + e];
        a[(int64_t)piv * m + e] = t;
        t = b[(int64_t)col * m + e];
        b[(int64_t)col * m + e] = b[(int64_t)piv * m + e];
        b[(int64_t)piv * m + e] = t;
      }
    __syncthreads();
    // scale the pivot row by 1 / pivot
    const cd p = a[(int64_t)col * m + col];
    const double pd2 = p.re * p.re + p.im * p.im;
    const cd ip = mk(p.re / pd2, -p.im / pd2);
    __syncthreads();
    for (int e = threadIdx.x; e < m; e += blockDim.x) {
      a[(int64_t)col * m + e] = a[(int64_t)col * m + e] * ip;
      b[(int64_t)col * m + e] = b[(int64_t)col * m + e] * ip;
    }
    // the column's factors, read before any row changes
    for (int r = threadIdx.x; r < m; r += blockDim.x) fac[r] = r == col ? mk(0.0, 0.0) : a[(int64_t)r * m + col];
    __syncthreads();
    // eliminate the column from every other row
    for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
      const int r = (int)(e / m), cc = (int)(e % m);
      if (r == col) continue;  // the pivot row is read, not written, in this step
      const cd f = fac[r];
      a[e] -= f * a[(int64_t)col * m + cc];
      b[e] -= f * b[(int64_t)col * m + cc];
    }
    __syncthreads();
  }
}

// Forward DFT over the slices of the signed periodic unknowns of column c:
// Xh[c][f][i] = sum_k sgn[k][i] v[idx[k][i]] exp(-2 pi i f k / R)
__global__ void k_circ_fwd(const cd* __restrict__ v, int64_t ld, const int32_t* __restrict__ idx,
                           const double* __restrict__ sgn, const cd* __restrict__ tw, int R, int m,
                           cd* __restrict__ Xh) {
  const int f = blockIdx.x, c = blockIdx.y;
  v += c * ld;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    cd acc = mk(0.0, 0.0);
    for (int k = 0; k < R; ++k) acc += (sgn[k * m + i] * v[idx[k * m + i]]) * twiddle(tw, (int64_t)f * k, R);
    Xh[((int64_t)c * R + f) * m + i] = acc;
  }
}

// Yh[c][f] = C_f^-1 Xh[c][f]
__global__ void k_circ_solve(const cd* __restrict__ inv, const cd* __restrict__ Xh, int R, int m,
                             cd* __restrict__ Yh) {
  extern __shared__ unsigned char smem_raw[];
  cd* xs = reinterpret_cast<cd*>(smem_raw);
  const int f = blockIdx.x, c = blockIdx.y;
  const cd* x = Xh + ((int64_t)c * R + f) * m;
  for (int j = threadIdx.x; j < m; j += blockDim.x) xs[j] = x[j];
  __syncthreads();
  const cd* M = inv + (int64_t)f * m * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    cd acc = mk(0.0, 0.0);
    for (int j = 0; j < m; ++j) cfma(acc, M[(int64_t)i * m + j], xs[j]);
    Yh[((int64_t)c * R + f) * m + i] = acc;
  }
}

// z[idx[k][i]] = sgn[k][i] (1/R) sum_f Yh[c][f][i] exp(+2 pi i f k / R)
__global__ void k_circ_inv(const cd* __restrict__ Yh, const int32_t* __restrict__ idx, const double* __restrict__ sgn,
                           const cd* __restrict__ tw, int R, int m, cd* __restrict__ z, int64_t ld) {
  const int k = blockIdx.x, c = blockIdx.y;
  z += c * ld;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    cd acc = mk(0.0, 0.0);
    for (int f = 0; f < R; ++f) acc += Yh[((int64_t)c * R + f) * m + i] * conj(twiddle(tw, (int64_t)f * k, R));
    z[idx[k * m + i]] = (sgn[k * m + i] / R) * acc;
  }
}

__global__ void k_circ_twiddles(cd* tw, int R) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= R) return;
  double sn, cs;
  sincospi(2.0 * k / R, &sn, &cs);
  tw[k] = mk(cs, -sn);
}

__global__ void k_unit_columns(void* X, int prec, int64_t N, int kb, const int32_t* __restrict__ idx,
                               const double* __restrict__ sgn, int row0) {
  const int j = threadIdx.x;
  if (j >= kb) return;
  const int64_t r = idx[row0 + j];
  if (prec == SCABEM_C128)
    reinterpret_cast<cd*>(X)[(int64_t)j * N + r] = mk(sgn[row0 + j], 0.0);
  else
    reinterpret_cast<cx<float>*>(X)[(int64_t)j * N + r] = mk((float)sgn[row0 + j], 0.0f);
}

void free_circ(Circulant& c) {
  cudaFree(c.idx);
  cudaFree(c.sgn);
  cudaFree(c.inv);
  cudaFree(c.work);
  cudaFree(c.tw);
  c = Circulant();
}

}  // namespace

void circulant_release(scabem_op* op) { free_circ(op->circ); }

int circulant_apply(scabem_op* op, const cd* in, cd* out, int k, int64_t cs_in, int64_t cs_out, cudaStream_t s) {
  Circulant& C = op->circ;
  for (int c0 = 0; c0 < k; c0 += KBATCH) {
    const int kc = std::min(KBATCH, k - c0);
    k_circ_fwd<<<dim3(C.R, kc), 128, 0, s>>>(in + c0 * cs_in, cs_in, C.idx, C.sgn, C.tw, C.R, C.m, C.work);
    CK(cudaGetLastError());
    cd* Yh = C.work + (int64_t)KBATCH * C.R * C.m;
    k_circ_solve<<<dim3(C.R, kc), 128, sizeof(cd) * C.m, s>>>(C.inv, C.work, C.R, C.m, Yh);
    CK(cudaGetLastError());
    k_circ_inv<<<dim3(C.R, kc), 128, 0, s>>>(Yh, C.idx, C.sgn, C.tw, C.R, C.m, out + c0 * cs_out, cs_out);
    CK(cudaGetLastError());
  }
  return SCABEM_OK;
}

int setup_circulant(scabem_op* op, const scabem_mesh* mesh, const scabem_circulant* P, cudaStream_t s) {
  free_circ(op->circ);
  if (P->count == 0) return SCABEM_OK;
  const int ax = P->axis, ay = (ax + 1) % 3, az = (ax + 2) % 3;
  const double dx = P->dx;
  const int first = P->first, R = P->count;
  // ---- slice layout of the plain-surface edges (host)
  auto vtx = [&](int64_t v, int a) { return mesh->V[3 * v + a]; };
  auto centroid = [&](int64_t t, int a) {
    return (vtx(mesh->T[3 * t], a) + vtx(mesh->T[3 * t + 1], a) + vtx(mesh->T[3 * t + 2], a)) / 3.0;
  };
  auto is_cap = [&](int64_t t) {
    double lo = 1e300, hi = -1e300;
    for (int k = 0; k < 3; ++k) {
      lo = std::min(lo, vtx(mesh->T[3 * t + k], ax));
      hi = std::max(hi, vtx(mesh->T[3 * t + k], ax));
    }
    return hi - lo < 1e-12 * dx;
  };
  struct Ent {
    std::array<double, 3> key;
    int64_t e;
  };
  std::vector<std::vector<Ent>> slices(R);
  for (int64_t e = 0; e < mesh->ne; ++e) {
    if (mesh->eclass[e] != 0) continue;
    const int64_t t0 = mesh->et[2 * e], t1 = mesh->et[2 * e + 1];
    if (is_cap(t0) || is_cap(t1)) continue;
    double mid[3];
    for (int a = 0; a < 3; ++a) mid[a] = 0.5 * (vtx(mesh->ev[2 * e], a) + vtx(mesh->ev[2 * e + 1], a));
    const double u = (mid[ax] - P->x0) / dx;
    const int64_t sl = (int64_t)std::floor(u + 1e-9);
    if (sl < first || sl >= first + R) continue;
    const double frac = std::round((u - sl) * 1e6) / 1e6;
    slices[sl - first].push_back({{frac, std::round(mid[ay] * 1e9) / 1e9, std::round(mid[az] * 1e9) / 1e9}, e});
  }
  const size_t me = slices[0].size();
  if (me == 0) {
    set_error("circulant preconditioner: no plain-surface edges in the first regular slice");
    return SCABEM_E_ARG;
  }
  for (auto& sv : slices) std::sort(sv.begin(), sv.end(), [](const Ent& a, const Ent& b) { return a.key < b.key; });
  const int m = (int)(2 * me);
  std::vector<int32_t> idx((size_t)R * m);
  std::vector<double> sgn((size_t)R * m);
  std::vector<std::array<double, 3>> ref(me);
  for (int k = 0; k < R; ++k) {
    if (slices[k].size() != me) {
      set_error("circulant preconditioner: slice " + std::to_string(first + k) + " is not a translate of slice " +
                std::to_string(first));
      return SCABEM_E_MESH;
    }
    for (size_t i = 0; i < me; ++i) {
      const int64_t e = slices[k][i].e;
      if (slices[k][i].key != slices[0][i].key) {
        set_error("circulant preconditioner: slice " + std::to_string(first + k) + " is not a translate of slice " +
                  std::to_string(first));
        return SCABEM_E_MESH;
      }
      double mid[3], plus[3], minus[3];
      for (int a = 0; a < 3; ++a) {
        mid[a] = 0.5 * (vtx(mesh->ev[2 * e], a) + vtx(mesh->ev[2 * e + 1], a));
        plus[a] = centroid(mesh->et[2 * e], a) - mid[a];
        minus[a] = centroid(mesh->et[2 * e + 1], a) - mid[a];
      }
      double sg = 1.0;
      if (k == 0) {
        for (int a = 0; a < 3; ++a) ref[i][a] = plus[a];
      } else {
        double dp = 0.0, dm = 0.0;
        for (int a = 0; a < 3; ++a) {
          dp += (plus[a] - ref[i][a]) * (plus[a] - ref[i][a]);
          dm += (minus[a] - ref[i][a]) * (minus[a] - ref[i][a]);
        }
        if (std::sqrt(dp) < 1e-9 * dx) sg = 1.0;
        else if (std::sqrt(dm) < 1e-9 * dx) sg = -1.0;
        else {
          set_error("circulant preconditioner: edge orientation does not repeat along the guide");
          return SCABEM_E_MESH;
        }
      }
      const int64_t ci = mesh->ecidx[e];
      idx[(size_t)k * m + i] = (int32_t)ci;                  // J^L
      idx[(size_t)k * m + me + i] = (int32_t)(mesh->nL + ci);  // M^L
      sgn[(size_t)k * m + i] = sg;
      sgn[(size_t)k * m + me + i] = sg;
    }
  }
  // ---- device tables
  Circulant& C = op->circ;
  C.R = R;
  C.m = m;
  auto fail = [&](int rc) {
    free_circ(C);
    return rc;
  };
  if (cudaMalloc(&C.idx, sizeof(int32_t) * R * m) != cudaSuccess ||
      cudaMalloc(&C.sgn, sizeof(double) * R * m) != cudaSuccess ||
      cudaMalloc(&C.inv, sizeof(cd) * (size_t)R * m * m) != cudaSuccess ||
      cudaMalloc(&C.work, sizeof(cd) * 2 * (size_t)KBATCH * R * m) != cudaSuccess ||
      cudaMalloc(&C.tw, sizeof(cd) * R) != cudaSuccess) {
    cudaGetLastError();
    set_error("circulant preconditioner: device allocation failed");
    return fail(SCABEM_E_NOMEM);
  }
  CK(cudaMemcpyAsync(C.idx, idx.data(), sizeof(int32_t) * R * m, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(C.sgn, sgn.data(), sizeof(double) * R * m, cudaMemcpyHostToDevice, s));
  k_circ_twiddles<<<(int)cdiv(R, 128), 128, 0, s>>>(C.tw, R);
  CK(cudaGetLastError());
  // ---- blocks from the operator's columns: the middle slice (Strang) or the
  // first and the last slice (Chan)
  const int prec = op->d.built ? SCABEM_C128 : SCABEM_C64;
  struct Pass {
    int src, mode;
  };
  std::vector<Pass> passes;
  if (P->kind == 1)
    passes = {{0, 1}, {R - 1, 2}};
  else
    passes = {{R / 2, 0}};
  const size_t csz = prec == SCABEM_C128 ? sizeof(cd) : sizeof(cx<float>);
  const int kb = std::min(KBATCH, m);
  if (kb > 1) {
    int rc = prec == SCABEM_C128 ? ensure_batch<double>(op, kb, s) : ensure_batch<float>(op, kb, s);
    if (rc) return fail(rc);
  }
  void *X = nullptr, *Y = nullptr;
  cd *cblk = nullptr, *Cf = nullptr;
  int* bad = nullptr;
  int rc = SCABEM_OK;
  do {
    if (cudaMalloc(&X, csz * op->N * kb) != cudaSuccess || cudaMalloc(&Y, csz * op->N * kb) != cudaSuccess ||
        cudaMalloc(&cblk, sizeof(cd) * (size_t)R * m * m) != cudaSuccess ||
        cudaMalloc(&Cf, sizeof(cd) * (size_t)R * m * m) != cudaSuccess || cudaMalloc(&bad, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      set_error("circulant preconditioner: device allocation failed");
      rc = SCABEM_E_NOMEM;
      break;
    }
    if (cudaMemsetAsync(cblk, 0, sizeof(cd) * (size_t)R * m * m, s) != cudaSuccess) {
      rc = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
      break;
    }
    for (const Pass& ps : passes)
      for (int j0 = 0; j0 < m && !rc; j0 += kb) {
        const int nb = std::min(kb, m - j0);
        if (cudaMemsetAsync(X, 0, csz * op->N * kb, s) != cudaSuccess) {
          rc = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
          break;
        }
        k_unit_columns<<<1, 32, 0, s>>>(X, prec, op->N, nb, C.idx, C.sgn, ps.src * m + j0);
        const unsigned gb = (unsigned)cdiv((int64_t)R * m * nb, 256);
        if (prec == SCABEM_C128) {
          rc = nb == 1 ? apply_one<double>(op, (const cd*)X, (cd*)Y, s)
                       : apply_batch<double>(op, (const cd*)X, op->N, (cd*)Y, op->N, nb, s);
          if (!rc)
            k_circ_gather<double><<<gb, 256, 0, s>>>((const cd*)Y, op->N, nb, j0, C.idx, C.sgn, R, m, ps.src, ps.mode,
                                                     cblk);
        } else {
          rc = nb == 1 ? apply_one<float>(op, (const cx<float>*)X, (cx<float>*)Y, s)
                       : apply_batch<float>(op, (const cx<float>*)X, op->N, (cx<float>*)Y, op->N, nb, s);
          if (!rc)
            k_circ_gather<float><<<gb, 256, 0, s>>>((const cx<float>*)Y, op->N, nb, j0, C.idx, C.sgn, R, m, ps.src,
                                                    ps.mode, cblk);
        }
      }
    if (rc) break;
    k_circ_dft_blocks<<<R, 256, 0, s>>>(cblk, C.tw, R, m, Cf);
    if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) {
      rc = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
      break;
    }
    if ((rc = set_max_smem(op->device, (const void*)k_circ_invert, (int)(sizeof(cd) * m)))) break;
    k_circ_invert<<<R, CIRC_THREADS, sizeof(cd) * m, s>>>(Cf, C.inv, m, bad);
    int hbad = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "circulant preconditioner set-up");
      break;
    }
    if (hbad) {
      set_error("circulant preconditioner: a DFT block of the circulant is singular");
      rc = SCABEM_E_BREAKDOWN;
    }
  } while (0);
  cudaFree(X);
  cudaFree(Y);
  cudaFree(cblk);
  cudaFree(Cf);
  cudaFree(bad);
  if (rc) return fail(rc);
  return SCABEM_OK;
}
