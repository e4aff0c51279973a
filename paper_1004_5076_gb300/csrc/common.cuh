// Internal declarations shared by the scabem translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/scabem.h"

// ------------------------------------------------------------------ complex
template <typename R>
struct __align__(2 * sizeof(R)) cx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) {
  cx<R> z;
  z.re = a;
  z.im = b;
  return z;
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a) { return mk(-a.re, -a.im); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mk(s * a.re, s * a.im); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, R s) { return mk(s * a.re, s * a.im); }
template <typename R>
__host__ __device__ __forceinline__ cx<R>& operator+=(cx<R>& a, cx<R> b) {
  a.re += b.re;
  a.im += b.im;
  return a;
}
template <typename R>
__host__ __device__ __forceinline__ cx<R>& operator-=(cx<R>& a, cx<R> b) {
  a.re -= b.re;
  a.im -= b.im;
  return a;
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> conj(cx<R> a) { return mk(a.re, -a.im); }
// multiply by j
template <typename R>
__host__ __device__ __forceinline__ cx<R> mulj(cx<R> a) { return mk(-a.im, a.re); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> czero() { return mk(R(0), R(0)); }
// a += s * b (s real)
template <typename R>
__host__ __device__ __forceinline__ void axpy(cx<R>& a, R s, cx<R> b) {
  a.re = fma(s, b.re, a.re);
  a.im = fma(s, b.im, a.im);
}
// a += b * c (complex)
template <typename R>
__host__ __device__ __forceinline__ void cfma(cx<R>& a, cx<R> b, cx<R> c) {
  a.re = fma(b.re, c.re, fma(-b.im, c.im, a.re));
  a.im = fma(b.re, c.im, fma(b.im, c.re, a.im));
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> cvt(cx<double> a) { return mk(R(a.re), R(a.im)); }

// A complex value as FP32 (hi, lo) pairs: re = rh + rl, im = ih + il, each
// lo at most half an ulp of its hi, so about 48 significant bits in the 16
// bytes of a complex128.  The GMRES basis is held this way: its products
// and sums then run on the FP32 units (exact products by FMA, compensated
// sums), which this GPU has some 75 times more of than FP64 units.
struct __align__(16) cdf {
  float rh, ih, rl, il;
};
__device__ __forceinline__ cx<double> df_join(cdf v) {
  return mk((double)v.rh + (double)v.rl, (double)v.ih + (double)v.il);
}
__device__ __forceinline__ cdf df_split(cx<double> v) {
  cdf o;
  o.rh = __double2float_rn(v.re);
  o.ih = __double2float_rn(v.im);
  o.rl = __double2float_rn(v.re - (double)o.rh);
  o.il = __double2float_rn(v.im - (double)o.ih);
  return o;
}

// small 3-vectors of complex
template <typename R>
struct cv3 {
  cx<R> x, y, z;
};

// ------------------------------------------------------------------ limits
constexpr int MAXQ = 7;    // quadrature points per triangle
constexpr int MAXP = 4;    // stencil points per axis
constexpr int NFIELD_IN = 12;
constexpr int NFIELD_OUT = 16;
constexpr int NREC = 20;   // per point and medium: A(3) phi gphi(3) curlA(3) F(3) psi gpsi(3) curlF(3)
constexpr int NCORR = 10;  // per point and medium: dP0, dP1(3), dQ(3), dC(3)
constexpr double ETA0 = 376.730313668;

// ------------------------------------------------------------------ profiling
// Stages of one apply: summaries (with the quadrature-point sources),
// projection, FFT axis 0 forward, (y, z) convolution with the Green
// function, FFT axis 0 inverse, points (interpolation, near field, testing
// and the row sums).
constexpr int NSTAGE = 6;
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;  // (NSTAGE + 1) per recorded apply
  int64_t used = 0;             // events recorded so far
};

// ------------------------------------------------------------------ handles
struct scabem_mesh {
  int64_t nv = 0, nt = 0, ne = 0, nL = 0, nR = 0, N = 0;
  std::vector<double> V;        // nv*3
  std::vector<int32_t> T;       // nt*3
  std::vector<int32_t> region;  // nt
  std::vector<int64_t> ev, et;  // ne*2
  std::vector<int32_t> eclass, ecidx;
  std::vector<int32_t> tri_edge, tri_sign;  // nt*3
  std::vector<double> elen;                 // ne
};

template <typename R>
struct PrecData {
  bool built = false;
  cx<R>* ghat[2] = {nullptr, nullptr};  // octant spectra [q0][q2][q1], scaled by 1/(P0 P1 P2)
  cx<R>* gt[2] = {nullptr, nullptr};    // transverse tables [q0][|d1|][|d2|] (direct mode)
  cx<R>* near = nullptr;                // [npairs][NCORR][q][2]
  cx<R>* tw[3] = {nullptr, nullptr, nullptr};  // forward twiddles per axis length
  R* L = nullptr;                       // Q * 3 * p stencil weights
  R* dL = nullptr;                      // Q * 3 * p derivative weights [1/um]
  R* sig = nullptr;                     // Q normalised conductivity
  R* tp = nullptr;                      // Q * 16 testing geometry: rel (3), w, X_k (3 x 3), div X_k (3)
  // workspaces
  cx<R>* summ = nullptr;  // nt * 3 sets * 4
  cx<R>* qsrc = nullptr;  // Q * 12 weighted point sources
  cx<R>* src = nullptr;   // 16 * n0 n1 n2 (12 sources; 16 in the transposed apply)
  cx<R>* stA = nullptr;   // 16 * P0 * cst (12 fields in the apply, 16 in the transposed apply)
  cx<R>* recb = nullptr;  // Q * 2 * NREC record adjoints (transposed apply)
  cx<R>* sbar = nullptr;  // 2 * nt * 12: summary adjoints (near + direct, total)
  cx<R>* nadj = nullptr;  // npairs * 12: per-pair near contributions (transposed apply)
  cx<R>* stB = nullptr;   // 16 * P0 * cst
  cx<R>* grid = nullptr;  // n0 n1 n2 * 16, point-major: [point][medium][J, M set][A or F (3), phi or psi]
  cx<R>* val = nullptr;   // nt * 3 * 4
  cx<R>* xs = nullptr;    // staging for host x/y: N * nrhs_cap
  cx<R>* ys = nullptr;
  int64_t stage_cap = 0;
  // right-hand sides the forward workspaces (summ, qsrc, src, stA, stB, grid)
  // hold side by side, at the column strides below
  int kcap = 1;
};

// Circulant preconditioner of the plain-surface block over R regular slices
// of m unknowns each (precond.cu); R = 0 when not set.
struct Circulant {
  int R = 0, m = 0;
  int32_t* idx = nullptr;     // R * m unknown indices, slice-major, in the common local order
  double* sgn = nullptr;      // R * m orientation signs
  cx<double>* inv = nullptr;  // R * m * m inverses of the DFT blocks of Strang's circulant
  cx<double>* work = nullptr;  // 2 * KBATCH * R * m spectra
  cx<double>* tw = nullptr;   // R twiddles exp(-2 pi i k / R)
};

struct scabem_op {
  int device = 0;
  int64_t nt = 0, ne = 0, N = 0, Q = 0, nL = 0, nR = 0;
  double ke = 0, ki = 0, ze = 1, zi = 1;
  int n[3] = {0, 0, 0}, P[3] = {0, 0, 0};
  double h = 0, origin[3] = {0, 0, 0};
  int p = 3, q = 6;
  double r_near = 0;
  int prec_mask = 0;
  // geometry (double)
  double* tri = nullptr;    // nt * 16: v0 v1 v2 c n area
  double* cX = nullptr;     // nt * 3: s_k l_k / (2 A)
  int32_t* unk = nullptr;   // nt * 3 (local k) * 3 (set): (index+1)*sign, 0 = none
  int32_t* region = nullptr;
  int32_t* trirow = nullptr;  // nt * 3 * 4: 1 if that (t,k,type) row exists
  int32_t* rowsrc = nullptr;  // N * 2 : ((t*3+k)*4+type) of T+ and T-
  int32_t* valrow = nullptr;  // nt * 12: row of each (t, k, type) value, -1 if none
  double* qp = nullptr;       // Q * 3
  double* qw = nullptr;       // Q
  int32_t* base = nullptr;    // Q * 3
  // projection as a gather over the ngnz grid points that some stencil
  // covers: point gpt[i] sums entries goff[i] .. goff[i+1]-1, entry e being
  // quadrature point gent[e] with stencil weight gwd[e] / gwf[e]; entries
  // are in (quadrature point, stencil slot) order within a grid point
  int64_t ngnz = 0;
  int32_t* gpt = nullptr;   // ngnz
  int32_t* goff = nullptr;  // ngnz + 1
  int32_t* gent = nullptr;  // Q * p^3
  double* gwd = nullptr;    // Q * p^3
  float* gwf = nullptr;     // Q * p^3
  double* gdd = nullptr;    // Q * p^3 * 3 derivative weights of the entries (transposed interpolation)
  float* gdf = nullptr;
  // columns (i1, i2) of the grid that some stencil covers, ascending: the
  // only ones whose sources are non-zero and whose potentials are read, so
  // the axis-0 transforms run on these alone; rowmask bit i1 is set when row
  // i1 holds one of them
  int64_t nac = 0;
  int32_t* acol = nullptr;  // nac
  uint64_t rowmask = 0;
  // (y, z) convolution: direct sum over the active columns (tdirect) with
  // gt[medium][q0][|d1|][|d2|] = (1/P0) x axis-0 transform of the spatial
  // Green table for |d1| < R1, |d2| < R2 (the active box), or 2-D FFT planes
  // with ghat.  acoord[j] = (i1 - b1) << 16 | (i2 - b2) of active column j.
  int transverse = 0;
  bool planes_fit = true;   // the (y, z) plane fits the 2-D FFT plane kernels
  bool direct_fits = true;  // the active columns fit one CTA of the direct (y, z) sums
  int a0_lines = 0;         // lines per CTA of the axis-0 transforms (0: the default rule)
  // columns per (field, k0) of the axis-0 intermediates stA, stB: the nac
  // active columns in order (compact) for the direct (y, z) sums, all n1 n2
  // for the FFT planes
  int64_t cst = 0;
  bool tdirect = false;
  int R1 = 0, R2 = 0;
  int32_t* acoord = nullptr;  // nac
  double* sig64 = nullptr;    // Q normalised (master copy)
  // near list
  int64_t npairs = 0;
  int32_t* noff = nullptr;  // nt + 1
  int32_t* nsrc = nullptr;  // npairs
  // reverse list: pairs rpair[roff[s] .. roff[s+1]) have source triangle s
  int32_t* roff = nullptr;   // nt + 1
  int32_t* rpair = nullptr;  // npairs
  // unknown -> up to 4 (triangle, local edge, set) uses, (code + 1) * sign,
  // code = (t * 3 + k) * 3 + set; 0 = unused (transposed current expansion)
  int32_t* xsrc = nullptr;   // N * 4
  cx<double>* gspatial[2] = {nullptr, nullptr};  // padded G tables, set-up only
  // per-edge block-diagonal preconditioner (exact self blocks, inverted)
  int32_t* etk = nullptr;   // ne * 4: T+, k+, T-, k-
  int32_t* ecls = nullptr;  // ne: 0 = plain, 1 = absorber
  int32_t* eunk = nullptr;  // ne * 3: unknown (= row) indices of the edge, -1 unused
  cx<double>* pinv = nullptr;  // ne * 9
  int precond_singular = 0;
  Circulant circ;
  PrecData<float> f;
  PrecData<double> d;
  int* err = nullptr;  // device error flag
  // set by a kernel whose bounded wait expired (host-mapped: readable
  // without a synchronisation; reported as SCABEM_E_TIMEOUT by the next call)
  int* tmo_h = nullptr;
  int* tmo_d = nullptr;
  Profiler prof;
};

// Column strides of the forward workspaces (complex values per right-hand side).
inline int64_t col_stride_grid(const scabem_op* op) {  // src and grid
  return (int64_t)NFIELD_OUT * op->n[0] * op->n[1] * op->n[2];
}
inline int64_t col_stride_st(const scabem_op* op) {  // stA and stB
  return (int64_t)NFIELD_OUT * op->P[0] * op->cst;
}
inline int64_t col_stride_summ(const scabem_op* op) { return op->nt * 12; }
inline int64_t col_stride_qsrc(const scabem_op* op) { return op->Q * 12; }
// Right-hand sides the batched apply handles per pass (one CTA of that many
// warps shares each target triangle's near-record stream).
constexpr int KBATCH = 8;

// Record the next stage-boundary event when profiling is on.
inline void prof_mark(scabem_op* op, cudaStream_t s) {
  Profiler& p = op->prof;
  if (p.on && p.used < (int64_t)p.ev.size()) cudaEventRecord(p.ev[p.used++], s);
}

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Raise a kernel's dynamic shared-memory limit on a device to at least
// `bytes`, calling the runtime only the first time a larger size is needed
// (the apply path then makes no attribute calls).
int set_max_smem(int device, const void* kernel, int bytes);
// One warp waits on an mbarrier that nothing completes, with the record
// rings' wait limit, and reports the expiry through op->tmo_d (synchronous).
int selftest_wait(scabem_op* op, cudaStream_t s);

// ------------------------------------------------------------------ launchers
// setup.cu
int setup_geometry(scabem_op* op, const scabem_mesh* m, cudaStream_t s);
int setup_green(scabem_op* op, cudaStream_t s);
int setup_near(scabem_op* op, cudaStream_t s);
int setup_sigma_monomial(scabem_op* op, int nseg, const double* seg, cudaStream_t s);
int setup_sigma_values(scabem_op* op, const double* per_q_host, cudaStream_t s);
int setup_sigma_bspline(scabem_op* op, double x0, double L, int axis, int ncoef, const double* coef, cudaStream_t s);
int setup_precond(scabem_op* op, cudaStream_t s);
int setup_gather(scabem_op* op, cudaStream_t s);
// k right-hand sides: column c of in / out starts at c * cs_in / c * cs_out
int precond_apply(scabem_op* op, const cx<double>* in, cx<double>* out, cudaStream_t s, bool transposed = false,
                  int k = 1, int64_t cs_in = 0, int64_t cs_out = 0);
// block-diagonal part only, from a basis held as FP32 (hi, lo) pairs, into
// complex64 (outf, the input of the complex64 operator) or complex128 (outd);
// SCABEM_E_ARG when a circulant block is set for this direction
int precond_apply_df(scabem_op* op, const cdf* in, cx<float>* outf, cx<double>* outd, cudaStream_t s,
                     bool transposed, int k, int64_t cs_in, int64_t cs_out);
bool precond_is_block_diagonal(const scabem_op* op, bool transposed);
// precond.cu
int setup_circulant(scabem_op* op, const scabem_mesh* mesh, const scabem_circulant* c, cudaStream_t s);
int circulant_apply(scabem_op* op, const cx<double>* in, cx<double>* out, int k, int64_t cs_in, int64_t cs_out,
                    cudaStream_t s);
void circulant_release(scabem_op* op);
// apply.cu
template <typename R>
int apply_one(scabem_op* op, const cx<R>* x, cx<R>* y, cudaStream_t s);
// y[:, c] = A x[:, c] for c < k <= pd.kcap (k <= KBATCH), x and y column-major with
// leading dimensions ldx, ldy; every stage runs once for all k columns and the
// point kernel reads each near record once for all of them
template <typename R>
int apply_batch(scabem_op* op, const cx<R>* x, int64_t ldx, cx<R>* y, int64_t ldy, int k, cudaStream_t s);
// grow the forward workspaces of precision R to k right-hand sides
template <typename R>
int ensure_batch(scabem_op* op, int k, cudaStream_t s);
// hs[p] = d(lam^T A x)/d sigma_p [per S] at every quadrature point (complex128)
int sigma_sensitivity_op(scabem_op* op, const cx<double>* x, const cx<double>* lam, cx<double>* hs,
                         cx<double>* yscr, cudaStream_t s);
// x_bar = A^T y_bar (transpose, no conjugation)
template <typename R>
int apply_adjoint_one(scabem_op* op, const cx<R>* ybar, cx<R>* xbar, cudaStream_t s);
// fft.cu
// adjoint = false: 12 sources -> 16 potentials (the apply); true: 16 -> 16,
// each field convolved with its medium's Green function (the transposed apply)
// ncol right-hand sides at once: column c of each workspace starts at
// c * col_stride_*(op) (the batched apply; ncol <= the batch capacity)
template <typename R>
int fft_conv(scabem_op* op, PrecData<R>& pd, cudaStream_t s, bool adjoint, int ncol = 1);
template <typename R>
int fft3d_full(scabem_op* op, cx<R>* data, const cx<R>* const tw[3], int dir, cudaStream_t s);
template <typename R>
int fft_axis_full(scabem_op* op, cx<R>* data, int axis, const cx<R>* tw, int dir, cudaStream_t s);
template <typename R>
int make_twiddles(cx<R>* tw, int len, cudaStream_t s);
// solve.cu
int rhs_impl(scabem_op* op, const scabem_source* src, int nsrc, void* b, int64_t ld, int prec, cudaStream_t s);
int sigma_gradient_impl(scabem_op* op, const cx<double>* x, const cx<double>* lam, const scabem_source* src, int nsrc,
                        const scabem_sigma* basis, double* g_out, cudaStream_t s);
int solve_impl(scabem_op* op, const void* b, void* x, int nrhs, int64_t ld, const scabem_solve_opts* o,
               cudaStream_t s, scabem_solve_info* info);
int fields_impl(scabem_op* op, const void* x, int nrhs, int64_t ld, const double* pts, int npts,
                const scabem_source* inc, double* E, cudaStream_t s);
int reflection_impl(scabem_op* op, const void* x, int nrhs, int64_t ld, const scabem_probe* pr,
                    const scabem_source* inc, double* out, cudaStream_t s);
int fields_eh_impl(scabem_op* op, const void* x, int nrhs, int64_t ld, const double* pts, int npts, int side,
                   const scabem_source* inc, double* E, double* H, cudaStream_t s);
int poynting_impl(scabem_op* op, const void* x, int nrhs, int64_t ld, const scabem_poynting* P,
                  const scabem_source* inc, double* out, cudaStream_t s);
int decay_fit_impl(const double* t, const double* E, int npts, double alo, double ahi, int na, double blo, double bhi,
                   int nb, double* out, cudaStream_t s);
int decay_rate_impl(scabem_op* op, const void* x, int nrhs, int64_t ld, const scabem_probe* pr, double alo,
                    double ahi, int na, const scabem_source* inc, double* out, cudaStream_t s);
