// C-ABI of the scabem library: handle management, argument validation, the
// RWG edge table (host topology), and dispatch to the device kernels.
#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "common.cuh"

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int set_max_smem(int device, const void* kernel, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> done;
  std::lock_guard<std::mutex> lock(mu);
  int& have = done[{device, kernel}];
  if (have >= bytes) return SCABEM_OK;
  CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  have = bytes;
  return SCABEM_OK;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return SCABEM_E_NOMEM;
  return SCABEM_E_DEVICE;
}

template <typename R>
int compute_summ(scabem_op* op, const cx<R>* x, cx<R>* summ, cudaStream_t s);

namespace {

int check_device() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  if (prop.major != 10 || prop.minor != 3) {
    set_error("this library is built for sm_103a (GB300) only; found compute capability " +
              std::to_string(prop.major) + "." + std::to_string(prop.minor));
    return SCABEM_E_DEVICE;
  }
  return SCABEM_OK;
}

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

template <typename T>
int dalloc(T** p, int64_t count) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)std::max<int64_t>(count, 1));
  if (e != cudaSuccess) {
    set_error(std::string("device allocation of ") + std::to_string(sizeof(T) * count) + " bytes failed");
    return SCABEM_E_NOMEM;
  }
  return SCABEM_OK;
}

#define TRY(x)                  \
  do {                          \
    int rc_ = (x);              \
    if (rc_ != SCABEM_OK) {     \
      scabem_op_destroy(op);    \
      return rc_;               \
    }                           \
  } while (0)

template <typename R>
void free_prec(PrecData<R>& pd) {
  cudaFree(pd.ghat[0]);
  cudaFree(pd.ghat[1]);
  cudaFree(pd.gt[0]);
  cudaFree(pd.gt[1]);
  cudaFree(pd.near);
  for (int a = 0; a < 3; ++a) cudaFree(pd.tw[a]);
  cudaFree(pd.L);
  cudaFree(pd.dL);
  cudaFree(pd.sig);
  cudaFree(pd.tp);
  cudaFree(pd.summ);
  cudaFree(pd.qsrc);
  cudaFree(pd.src);
  cudaFree(pd.stA);
  cudaFree(pd.stB);
  cudaFree(pd.grid);
  cudaFree(pd.val);
  cudaFree(pd.recb);
  cudaFree(pd.nadj);
  cudaFree(pd.sbar);
  cudaFree(pd.xs);
  cudaFree(pd.ys);
  pd = PrecData<R>();
}

// The axis-0 intermediates, once the active columns and the (y, z) mode are
// known: compact (active columns only) for the direct sums, whole planes for
// the FFT planes; the axis-0 transform writes only the active columns, so
// the rest of a whole plane stays zero from here.
template <typename R>
int alloc_st(scabem_op* op, PrecData<R>& pd, cudaStream_t s) {
  if (!pd.built) return SCABEM_OK;
  const int64_t n = col_stride_st(op);
  int rc;
  if ((rc = dalloc(&pd.stA, n)) || (rc = dalloc(&pd.stB, n))) return rc;
  CK(cudaMemsetAsync(pd.stA, 0, sizeof(cx<R>) * n, s));
  CK(cudaMemsetAsync(pd.stB, 0, sizeof(cx<R>) * n, s));
  return SCABEM_OK;
}

template <typename R>
int alloc_prec(scabem_op* op, PrecData<R>& pd, bool workspaces, cudaStream_t s) {
  int rc;
  if ((rc = dalloc(&pd.L, op->Q * 3 * op->p))) return rc;
  if ((rc = dalloc(&pd.dL, op->Q * 3 * op->p))) return rc;
  if ((rc = dalloc(&pd.sig, op->Q))) return rc;
  if ((rc = dalloc(&pd.tp, op->Q * 16))) return rc;
  if (!workspaces) return SCABEM_OK;
  const int64_t ng = (int64_t)op->n[0] * op->n[1] * op->n[2];
  for (int a = 0; a < 3; ++a) {
    if ((rc = dalloc(&pd.tw[a], op->P[a]))) return rc;
    if ((rc = make_twiddles<R>(pd.tw[a], op->P[a], s))) return rc;
  }
  if ((rc = dalloc(&pd.summ, op->nt * 12))) return rc;
  if ((rc = dalloc(&pd.qsrc, op->Q * 12))) return rc;
  if ((rc = dalloc(&pd.src, NFIELD_OUT * ng))) return rc;
  // grid points no stencil covers are never written by the projection
  CK(cudaMemsetAsync(pd.src, 0, sizeof(cx<R>) * NFIELD_OUT * ng, s));
  if ((rc = dalloc(&pd.recb, op->Q * 2 * NREC))) return rc;
  if ((rc = dalloc(&pd.sbar, 2 * op->nt * 12))) return rc;
  if ((rc = dalloc(&pd.grid, NFIELD_OUT * ng))) return rc;
  if ((rc = dalloc(&pd.val, op->nt * 12))) return rc;
  pd.built = true;
  return SCABEM_OK;
}

}  // namespace

// Grow the forward workspaces of one precision to k right-hand sides side by
// side (column c at c * col_stride_*): the summaries, point sources, source
// grids, axis-0 intermediates and potential grids.  New source grids and
// intermediates start at zero (stencils and active columns leave the rest
// untouched), as at creation.
template <typename R>
int ensure_batch(scabem_op* op, int k, cudaStream_t s) {
  PrecData<R>& pd = *reinterpret_cast<PrecData<R>*>(sizeof(R) == 4 ? (void*)&op->f : (void*)&op->d);
  if (!pd.built) {
    set_error("operator was not built for this precision (prec_mask)");
    return SCABEM_E_ARG;
  }
  if (k <= pd.kcap) return SCABEM_OK;
  CK(cudaStreamSynchronize(s));  // nothing in flight uses the old buffers
  cx<R>* nb[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  cx<R>** cur[6] = {&pd.summ, &pd.qsrc, &pd.src, &pd.stA, &pd.stB, &pd.grid};
  const int64_t cs[6] = {col_stride_summ(op), col_stride_qsrc(op), col_stride_grid(op), col_stride_st(op),
                         col_stride_st(op), col_stride_grid(op)};
  for (int i = 0; i < 6; ++i) {
    int rc = dalloc(&nb[i], cs[i] * k);
    if (rc) {
      for (int j = 0; j < i; ++j) cudaFree(nb[j]);
      return rc;
    }
  }
  // column 0 keeps its contents (the single-column paths use it); the others start at zero
  for (int i = 0; i < 6; ++i) {
    CK(cudaMemcpyAsync(nb[i], *cur[i], sizeof(cx<R>) * cs[i], cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(nb[i] + cs[i], 0, sizeof(cx<R>) * cs[i] * (k - 1), s));
  }
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < 6; ++i) {
    cudaFree(*cur[i]);
    *cur[i] = nb[i];
  }
  pd.kcap = k;
  return SCABEM_OK;
}
template int ensure_batch<float>(scabem_op*, int, cudaStream_t);
template int ensure_batch<double>(scabem_op*, int, cudaStream_t);

namespace {

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Stage host x on the device when needed, then run fn(device x).
template <typename F>
int with_device_x(scabem_op* op, const void* x, int nrhs, int64_t ld, cudaStream_t s, F fn) {
  if (is_device_ptr(x)) return fn(x);
  void* dx = nullptr;
  const size_t bytes = sizeof(cx<double>) * ld * nrhs;
  CK(cudaMalloc(&dx, bytes));
  CK(cudaMemcpyAsync(dx, x, bytes, cudaMemcpyHostToDevice, s));
  const int rc = fn(dx);
  cudaStreamSynchronize(s);
  cudaFree(dx);
  return rc;
}

template <typename R>
int apply_col(scabem_op* op, const cx<R>* x, cx<R>* y, bool adjoint, cudaStream_t s) {
  return adjoint ? apply_adjoint_one<R>(op, x, y, s) : apply_one<R>(op, x, y, s);
}

template <typename R>
int apply_prec(scabem_op* op, const void* xv, void* yv, int nrhs, int64_t ld, cudaStream_t s, bool adjoint) {
  PrecData<R>& pd = *reinterpret_cast<PrecData<R>*>(sizeof(R) == 4 ? (void*)&op->f : (void*)&op->d);
  if (!pd.built) {
    set_error("operator was not built for this precision (prec_mask)");
    return SCABEM_E_ARG;
  }
  const bool xd = is_device_ptr(xv), yd = is_device_ptr(yv);
  const int64_t N = op->N;
  if (!adjoint && nrhs > 1) {
    // batches of up to KBATCH columns: each stage runs once per batch and the
    // point kernel reads the near records once per batch
    const int kb = nrhs < KBATCH ? nrhs : KBATCH;
    int rc = ensure_batch<R>(op, kb, s);
    if (rc) return rc;
    if (!xd || !yd) {
      if (pd.stage_cap < N * kb) {
        cudaFree(pd.xs);
        cudaFree(pd.ys);
        pd.xs = pd.ys = nullptr;
        pd.stage_cap = 0;
        if ((rc = dalloc(&pd.xs, N * kb)) || (rc = dalloc(&pd.ys, N * kb))) return rc;
        pd.stage_cap = N * kb;
      }
    }
    for (int c0 = 0; c0 < nrhs; c0 += kb) {
      const int k = nrhs - c0 < kb ? nrhs - c0 : kb;
      const cx<R>* xin = (const cx<R>*)xv + c0 * ld;
      int64_t ldx = ld, ldy = ld;
      if (!xd) {
        for (int c = 0; c < k; ++c)
          CK(cudaMemcpyAsync(pd.xs + c * N, xin + c * ld, sizeof(cx<R>) * N, cudaMemcpyHostToDevice, s));
        xin = pd.xs;
        ldx = N;
      }
      cx<R>* yout = yd ? (cx<R>*)yv + c0 * ld : pd.ys;
      if (!yd) ldy = N;
      rc = apply_batch<R>(op, xin, ldx, yout, ldy, k, s);
      if (rc) return rc;
      if (!yd)
        for (int c = 0; c < k; ++c)
          CK(cudaMemcpyAsync((cx<R>*)yv + (c0 + c) * ld, pd.ys + c * N, sizeof(cx<R>) * N, cudaMemcpyDeviceToHost,
                             s));
    }
    if (!xd || !yd) CK(cudaStreamSynchronize(s));
    return SCABEM_OK;
  }
  if (xd && yd) {
    for (int c = 0; c < nrhs; ++c) {
      int rc = apply_col<R>(op, (const cx<R>*)xv + c * ld, (cx<R>*)yv + c * ld, adjoint, s);
      if (rc) return rc;
    }
    return SCABEM_OK;
  }
  if (pd.stage_cap < N) {
    cudaFree(pd.xs);
    cudaFree(pd.ys);
    pd.xs = pd.ys = nullptr;
    int rc;
    if ((rc = dalloc(&pd.xs, N)) || (rc = dalloc(&pd.ys, N))) return rc;
    pd.stage_cap = N;
  }
  for (int c = 0; c < nrhs; ++c) {
    const cx<R>* xc = (const cx<R>*)xv + c * ld;
    cx<R>* yc = (cx<R>*)yv + c * ld;
    const cx<R>* xin = xc;
    if (!xd) {
      CK(cudaMemcpyAsync(pd.xs, xc, sizeof(cx<R>) * N, cudaMemcpyHostToDevice, s));
      xin = pd.xs;
    }
    cx<R>* yout = yd ? yc : pd.ys;
    int rc = apply_col<R>(op, xin, yout, adjoint, s);
    if (rc) return rc;
    if (!yd) CK(cudaMemcpyAsync(yc, pd.ys, sizeof(cx<R>) * N, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  return SCABEM_OK;
}

}  // namespace

extern "C" {

const char* scabem_last_error(void) { return g_last_error.c_str(); }

int scabem_mesh_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, const int32_t* region,
                       scabem_mesh_t* out) {
  if (!out || !xyz || !tri || !region || nv < 3 || nt < 2) {
    set_error("scabem_mesh_create: null pointer or too few vertices/triangles");
    return SCABEM_E_ARG;
  }
  if (nt > INT32_MAX / 8 || nv > INT32_MAX / 2) {
    set_error("scabem_mesh_create: mesh too large");
    return SCABEM_E_ARG;
  }
  *out = nullptr;
  scabem_mesh* m = new (std::nothrow) scabem_mesh();
  if (!m) {
    set_error("host allocation failed");
    return SCABEM_E_NOMEM;
  }
  m->nv = nv;
  m->nt = nt;
  m->V.assign(xyz, xyz + 3 * nv);
  m->T.assign(tri, tri + 3 * nt);
  m->region.assign(region, region + nt);
  for (int64_t i = 0; i < 3 * nv; ++i)
    if (!std::isfinite(m->V[i])) {
      set_error("non-finite vertex coordinate");
      delete m;
      return SCABEM_E_NONFINITE;
    }
  for (int64_t t = 0; t < nt; ++t) {
    if (m->region[t] != 0 && m->region[t] != 1) {
      set_error("region flags must be 0 or 1");
      delete m;
      return SCABEM_E_ARG;
    }
    int32_t a = m->T[3 * t], b = m->T[3 * t + 1], c = m->T[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv || a == b || b == c || a == c) {
      set_error("triangle " + std::to_string(t) + " has invalid vertex indices");
      delete m;
      return SCABEM_E_MESH;
    }
    const double* p0 = &m->V[3 * a];
    const double* p1 = &m->V[3 * b];
    const double* p2 = &m->V[3 * c];
    double u[3], v[3];
    for (int k = 0; k < 3; ++k) {
      u[k] = p1[k] - p0[k];
      v[k] = p2[k] - p0[k];
    }
    const double cx_ = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
    if (!(cx_ * cx_ + cy * cy + cz * cz > 0)) {
      set_error("triangle " + std::to_string(t) + " is degenerate (zero area)");
      delete m;
      return SCABEM_E_MESH;
    }
  }
  // directed edges: local edge k runs from vertex k+1 to vertex k+2
  std::unordered_map<uint64_t, int64_t> dir;
  dir.reserve((size_t)(3 * nt * 2));
  const uint64_t NV = (uint64_t)nv;
  for (int64_t t = 0; t < nt; ++t)
    for (int k = 0; k < 3; ++k) {
      const uint64_t u = (uint64_t)m->T[3 * t + (k + 1) % 3], w = (uint64_t)m->T[3 * t + (k + 2) % 3];
      if (!dir.emplace(u * NV + w, 3 * t + k).second) {
        set_error("non-manifold or inconsistently oriented mesh (directed edge used twice)");
        delete m;
        return SCABEM_E_MESH;
      }
    }
  std::vector<uint64_t> keys;
  keys.reserve(dir.size() / 2 + 1);
  for (auto& kv : dir) {
    const uint64_t u = kv.first / NV, w = kv.first % NV;
    if (u < w) keys.push_back(kv.first);
  }
  std::sort(keys.begin(), keys.end());
  const int64_t ne = (int64_t)keys.size();
  if (2 * ne != 3 * nt) {
    set_error("open mesh: every edge must be shared by exactly two triangles");
    delete m;
    return SCABEM_E_MESH;
  }
  m->ne = ne;
  m->ev.resize(2 * ne);
  m->et.resize(2 * ne);
  m->eclass.resize(ne);
  m->ecidx.resize(ne);
  m->elen.resize(ne);
  m->tri_edge.assign(3 * nt, -1);
  m->tri_sign.assign(3 * nt, 0);
  for (int64_t e = 0; e < ne; ++e) {
    const uint64_t u = keys[e] / NV, w = keys[e] % NV;
    auto fp = dir.find(u * NV + w);
    auto fm = dir.find(w * NV + u);
    if (fm == dir.end()) {
      set_error("open mesh: every edge must be shared by exactly two triangles");
      delete m;
      return SCABEM_E_MESH;
    }
    const int64_t tp = fp->second / 3, kp = fp->second % 3, tm = fm->second / 3, km = fm->second % 3;
    m->ev[2 * e] = (int64_t)u;
    m->ev[2 * e + 1] = (int64_t)w;
    m->et[2 * e] = tp;
    m->et[2 * e + 1] = tm;
    m->tri_edge[3 * tp + kp] = (int32_t)e;
    m->tri_sign[3 * tp + kp] = 1;
    m->tri_edge[3 * tm + km] = (int32_t)e;
    m->tri_sign[3 * tm + km] = -1;
    m->eclass[e] = (m->region[tp] == 1 && m->region[tm] == 1) ? 1 : 0;
    double d2 = 0;
    for (int k = 0; k < 3; ++k) {
      const double dd = m->V[3 * w + k] - m->V[3 * u + k];
      d2 += dd * dd;
    }
    m->elen[e] = std::sqrt(d2);
  }
  int64_t cnt[2] = {0, 0};
  for (int64_t e = 0; e < ne; ++e) m->ecidx[e] = (int32_t)cnt[m->eclass[e]]++;
  m->nL = cnt[0];
  m->nR = cnt[1];
  m->N = 2 * m->nL + 3 * m->nR;
  if (m->N > INT32_MAX / 2) {
    set_error("too many unknowns");
    delete m;
    return SCABEM_E_ARG;
  }
  *out = m;
  return SCABEM_OK;
}

int scabem_mesh_info(scabem_mesh_t m, int64_t* nL, int64_t* nR, int64_t* N) {
  if (!m) {
    set_error("null mesh");
    return SCABEM_E_ARG;
  }
  if (nL) *nL = m->nL;
  if (nR) *nR = m->nR;
  if (N) *N = m->N;
  return SCABEM_OK;
}

int scabem_mesh_edges(scabem_mesh_t m, int64_t* edge_v, int64_t* edge_t, int32_t* edge_class) {
  if (!m) {
    set_error("null mesh");
    return SCABEM_E_ARG;
  }
  if (edge_v) std::memcpy(edge_v, m->ev.data(), sizeof(int64_t) * 2 * m->ne);
  if (edge_t) std::memcpy(edge_t, m->et.data(), sizeof(int64_t) * 2 * m->ne);
  if (edge_class) std::memcpy(edge_class, m->eclass.data(), sizeof(int32_t) * m->ne);
  return SCABEM_OK;
}

void scabem_mesh_destroy(scabem_mesh_t m) { delete m; }

int scabem_op_create(scabem_mesh_t m, const scabem_media* md, const scabem_grid_opts* o, void* stream,
                     scabem_op_t* out) {
  if (!m || !md || !o || !out) {
    set_error("scabem_op_create: null argument");
    return SCABEM_E_ARG;
  }
  *out = nullptr;
  int rc = check_device();
  if (rc) return rc;
  const double vals[5] = {md->eps_i, md->mu_i, md->eps_e, md->mu_e, md->lambda0};
  for (double v : vals)
    if (!(v > 0) || !std::isfinite(v)) {
      set_error("media parameters and wavelength must be finite and positive");
      return SCABEM_E_ARG;
    }
  if (!pow2_in(2 * o->n[0], 8, 1024) || !pow2_in(2 * o->n[1], 8, 512) || !pow2_in(2 * o->n[2], 8, 512)) {
    set_error("grid: 2*n must be a power of two, in [8, 1024] along x and in [8, 512] along y and z");
    return SCABEM_E_ARG;
  }
  // the 2-D FFT plane kernels hold a whole (y, z) plane in shared memory
  const bool planes_fit = 2 * o->n[1] <= 128 && 2 * o->n[2] <= 128 && 4 * o->n[1] * o->n[2] <= 4096;
  if (!planes_fit && o->transverse == 1) {
    set_error("grid: the FFT (y, z) planes need 2 n_y, 2 n_z <= 128 and (2 n_y)(2 n_z) <= 4096; larger planes "
              "run as direct sums (transverse = 2 or 0)");
    return SCABEM_E_ARG;
  }
  if (o->p < 2 || o->p > MAXP || !(o->q == 1 || o->q == 3 || o->q == 6 || o->q == 7) || !(o->h > 0) ||
      !(o->r_near >= 0) || o->prec_mask < 1 || o->prec_mask > 3 || o->transverse < 0 || o->transverse > 2) {
    set_error("grid options: need p in 2..4, q in {1,3,6,7}, h > 0, r_near >= 0, prec_mask in 1..3, "
              "transverse in 0..2");
    return SCABEM_E_ARG;
  }
  scabem_op* op = new (std::nothrow) scabem_op();
  if (!op) {
    set_error("host allocation failed");
    return SCABEM_E_NOMEM;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaGetDevice(&op->device);
  op->nt = m->nt;
  op->ne = m->ne;
  op->N = m->N;
  op->nL = m->nL;
  op->nR = m->nR;
  op->q = o->q;
  op->p = o->p;
  op->Q = m->nt * o->q;
  op->h = o->h;
  op->r_near = o->r_near;
  op->prec_mask = o->prec_mask;
  op->transverse = o->transverse;
  op->planes_fit = planes_fit;
  for (int a = 0; a < 3; ++a) {
    op->n[a] = o->n[a];
    op->P[a] = 2 * o->n[a];
    op->origin[a] = o->origin[a];
  }
  const double w = 2.0 * M_PI / md->lambda0;
  op->ke = w * std::sqrt(md->eps_e * md->mu_e);
  op->ki = w * std::sqrt(md->eps_i * md->mu_i);
  op->ze = std::sqrt(md->mu_e / md->eps_e);
  op->zi = std::sqrt(md->mu_i / md->eps_i);

  // host tables: unknown codes per (triangle, local edge, set) and row sources
  std::vector<int32_t> unk(9 * m->nt, 0), rowsrc(2 * m->N, 0);
  const int64_t nL = m->nL, nR = m->nR;
  for (int64_t t = 0; t < m->nt; ++t)
    for (int k = 0; k < 3; ++k) {
      const int32_t e = m->tri_edge[3 * t + k];
      const int64_t ci = m->ecidx[e];
      int32_t* u = &unk[(3 * t + k) * 3];
      if (m->eclass[e] == 0) {
        u[0] = (int32_t)(ci + 1);
        u[1] = -(int32_t)(ci + 1);
        u[2] = (int32_t)(nL + ci + 1);
      } else {
        u[0] = (int32_t)(2 * nL + ci + 1);
        u[1] = (int32_t)(2 * nL + nR + ci + 1);
        u[2] = (int32_t)(2 * nL + 2 * nR + ci + 1);
      }
    }
  for (int64_t e = 0; e < m->ne; ++e) {
    int64_t src[2];
    for (int side = 0; side < 2; ++side) {
      const int64_t t = m->et[2 * e + side];
      int kk = 0;
      while (m->tri_edge[3 * t + kk] != e) ++kk;
      src[side] = (t * 3 + kk) * 4;
    }
    const int64_t ci = m->ecidx[e];
    if (m->eclass[e] == 0) {
      const int64_t r0 = ci, r1 = nL + ci;
      rowsrc[2 * r0] = (int32_t)(src[0] + 0);
      rowsrc[2 * r0 + 1] = (int32_t)(src[1] + 0);
      rowsrc[2 * r1] = (int32_t)(src[0] + 1);
      rowsrc[2 * r1 + 1] = (int32_t)(src[1] + 1);
    } else {
      const int64_t r0 = 2 * nL + ci, r2 = 2 * nL + nR + ci, r3 = 2 * nL + 2 * nR + ci;
      rowsrc[2 * r0] = (int32_t)(src[0] + 0);
      rowsrc[2 * r0 + 1] = (int32_t)(src[1] + 0);
      rowsrc[2 * r2] = (int32_t)(src[0] + 2);
      rowsrc[2 * r2 + 1] = (int32_t)(src[1] + 2);
      rowsrc[2 * r3] = (int32_t)(src[0] + 3);
      rowsrc[2 * r3 + 1] = (int32_t)(src[1] + 3);
    }
  }
  // uses of each unknown in the current expansion (transposed apply)
  std::vector<int32_t> xsrc(4 * m->N, 0);
  {
    std::vector<int> nuse(m->N, 0);
    for (int64_t t = 0; t < m->nt; ++t)
      for (int k = 0; k < 3; ++k)
        for (int set = 0; set < 3; ++set) {
          const int32_t u = unk[(3 * t + k) * 3 + set];
          if (u == 0) continue;
          const int64_t idx = (u > 0 ? u : -u) - 1;
          const int32_t code = (int32_t)((t * 3 + k) * 3 + set) + 1;
          if (nuse[idx] < 4) xsrc[4 * idx + nuse[idx]] = u > 0 ? code : -code;
          ++nuse[idx];
        }
    for (int64_t i = 0; i < m->N; ++i)
      if (nuse[i] > 4) {
        set_error("internal: an unknown has more than four current uses");
        scabem_op_destroy(op);
        return SCABEM_E_MESH;
      }
  }
  // row of each (triangle, local edge, type) tested value, -1 if none
  std::vector<int32_t> valrow(12 * m->nt, -1);
  for (int64_t r = 0; r < m->N; ++r) {
    valrow[rowsrc[2 * r]] = (int32_t)r;
    valrow[rowsrc[2 * r + 1]] = (int32_t)r;
  }
  std::vector<int32_t> etk(4 * m->ne), ecls(m->ne), eunk(3 * m->ne, -1);
  for (int64_t e = 0; e < m->ne; ++e) {
    for (int side = 0; side < 2; ++side) {
      const int64_t t = m->et[2 * e + side];
      int kk = 0;
      while (m->tri_edge[3 * t + kk] != e) ++kk;
      etk[4 * e + 2 * side] = (int32_t)t;
      etk[4 * e + 2 * side + 1] = kk;
    }
    ecls[e] = m->eclass[e];
    const int64_t ci = m->ecidx[e];
    if (m->eclass[e] == 0) {
      eunk[3 * e] = (int32_t)ci;
      eunk[3 * e + 1] = (int32_t)(nL + ci);
    } else {
      eunk[3 * e] = (int32_t)(2 * nL + ci);
      eunk[3 * e + 1] = (int32_t)(2 * nL + nR + ci);
      eunk[3 * e + 2] = (int32_t)(2 * nL + 2 * nR + ci);
    }
  }
  TRY(dalloc(&op->etk, 4 * op->ne));
  TRY(dalloc(&op->ecls, op->ne));
  TRY(dalloc(&op->eunk, 3 * op->ne));
  TRY(dalloc(&op->pinv, 9 * op->ne));
  TRY(dalloc(&op->tri, 16 * op->nt));
  TRY(dalloc(&op->cX, 3 * op->nt));
  TRY(dalloc(&op->unk, 9 * op->nt));
  TRY(dalloc(&op->region, op->nt));
  TRY(dalloc(&op->rowsrc, 2 * op->N));
  TRY(dalloc(&op->valrow, 12 * op->nt));
  TRY(dalloc(&op->xsrc, 4 * op->N));
  TRY(dalloc(&op->qp, 3 * op->Q));
  TRY(dalloc(&op->qw, op->Q));
  TRY(dalloc(&op->base, 3 * op->Q));
  TRY(dalloc(&op->sig64, op->Q));
  TRY(dalloc(&op->err, 1));
  TRY(cudaHostAlloc(&op->tmo_h, sizeof(int), cudaHostAllocMapped) == cudaSuccess ? SCABEM_OK : SCABEM_E_NOMEM);
  *op->tmo_h = 0;
  TRY(cudaHostGetDevicePointer(&op->tmo_d, op->tmo_h, 0) == cudaSuccess ? SCABEM_OK : SCABEM_E_DEVICE);
  TRY(alloc_prec(op, op->d, (op->prec_mask & 2) != 0, s));
  TRY(alloc_prec(op, op->f, (op->prec_mask & 1) != 0, s));
  auto upload = [&](void* dst, const void* src, size_t bytes) -> int {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? SCABEM_OK : cuda_fail(e, "cudaMemcpyAsync (host tables)");
  };
  TRY(upload(op->unk, unk.data(), sizeof(int32_t) * unk.size()));
  TRY(upload(op->rowsrc, rowsrc.data(), sizeof(int32_t) * rowsrc.size()));
  TRY(upload(op->valrow, valrow.data(), sizeof(int32_t) * valrow.size()));
  TRY(upload(op->xsrc, xsrc.data(), sizeof(int32_t) * xsrc.size()));
  TRY(upload(op->region, m->region.data(), sizeof(int32_t) * m->nt));
  TRY(upload(op->etk, etk.data(), sizeof(int32_t) * etk.size()));
  TRY(upload(op->ecls, ecls.data(), sizeof(int32_t) * ecls.size()));
  TRY(upload(op->eunk, eunk.data(), sizeof(int32_t) * eunk.size()));
  TRY(setup_geometry(op, m, s));
  TRY(setup_gather(op, s));
  op->cst = op->tdirect ? op->nac : (int64_t)op->n[1] * op->n[2];
  TRY(alloc_st(op, op->d, s));
  TRY(alloc_st(op, op->f, s));
  TRY(setup_green(op, s));
  TRY(setup_near(op, s));
  TRY(setup_sigma_monomial(op, 0, nullptr, s));
  *out = op;
  return SCABEM_OK;
}

int scabem_op_info(scabem_op_t op, int64_t* npairs, int64_t* b64, int64_t* b128, int64_t* nq) {
  if (!op) {
    set_error("null operator");
    return SCABEM_E_ARG;
  }
  const int64_t rec = op->npairs * op->q * 2 * NCORR;
  if (npairs) *npairs = op->npairs;
  if (b64) *b64 = rec * (int64_t)sizeof(cx<float>);
  if (b128) *b128 = rec * (int64_t)sizeof(cx<double>);
  if (nq) *nq = op->Q;
  return SCABEM_OK;
}

int scabem_grid_plan(scabem_mesh_t mesh, double h_max, int32_t p, double near_h, scabem_grid_opts* opts) {
  if (!mesh || !opts || !(h_max > 0.0) || !std::isfinite(h_max) || p < 2 || p > MAXP || !(near_h >= 0.0) ||
      !std::isfinite(near_h) || mesh->nv < 1) {
    set_error("scabem_grid_plan: null argument, h_max <= 0, p outside 2..4 or near_h < 0");
    return SCABEM_E_ARG;
  }
  double lo[3], hi[3];
  for (int a = 0; a < 3; ++a) lo[a] = hi[a] = mesh->V[a];
  for (int64_t v = 1; v < mesh->nv; ++v)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], mesh->V[3 * v + a]);
      hi[a] = std::max(hi[a], mesh->V[3 * v + a]);
    }
  // usable stencil-base range on an axis of n points: u in [(p-2)/2, n - p/2), n - p + 1 cells;
  // the mesh gets n - p - 1.5 of them, 1.25 cells of slack on either side
  const int tmax[3] = {1024, 128, 128};
  int n[3];
  for (int a = 0; a < 3; ++a) {
    const double need = (hi[a] - lo[a]) / h_max + p + 1.5;
    int t = 8;
    while (t < 2 * need && t <= tmax[a]) t *= 2;
    if (t > tmax[a]) {
      set_error("scabem_grid_plan: h_max too small for the transform limits along axis " + std::to_string(a));
      return SCABEM_E_ARG;
    }
    n[a] = t / 2;
  }
  if (4 * n[1] * n[2] > 4096) {
    set_error("scabem_grid_plan: h_max too small for the (y, z) plane limit (2 n_y)(2 n_z) <= 4096");
    return SCABEM_E_ARG;
  }
  double h = 0.0;
  for (int a = 0; a < 3; ++a) h = std::max(h, (hi[a] - lo[a]) / (n[a] - p - 1.5));
  if (!(h > 0.0)) h = h_max;
  // small fractions of a cell keep the points of structured meshes off cell boundaries
  const double off[3] = {0.0731, 0.0419, 0.0257};
  for (int a = 0; a < 3; ++a) {
    opts->n[a] = n[a];
    opts->origin[a] = 0.5 * (lo[a] + hi[a]) - h * (0.5 * (n[a] - 1) - off[a]);
  }
  opts->h = h;
  opts->p = p;
  opts->q = 6;
  opts->r_near = near_h * h;
  opts->prec_mask = 3;
  opts->transverse = 0;
  return SCABEM_OK;
}

int scabem_op_grid_info(scabem_op_t op, int64_t* npts, int64_t* ncols, int32_t* direct) {
  if (!op) {
    set_error("null operator");
    return SCABEM_E_ARG;
  }
  if (npts) *npts = op->ngnz;
  if (ncols) *ncols = op->nac;
  if (direct) *direct = op->tdirect ? 1 : 0;
  return SCABEM_OK;
}

int scabem_profile(scabem_op_t op, int32_t enable, int32_t max_applies) {
  if (!op || (enable && max_applies < 1)) {
    set_error("scabem_profile: null operator or max_applies < 1");
    return SCABEM_E_ARG;
  }
  Profiler& p = op->prof;
  for (auto e : p.ev) cudaEventDestroy(e);
  p.ev.clear();
  p.used = 0;
  p.on = false;
  if (!enable) return SCABEM_OK;
  p.ev.resize((size_t)(NSTAGE + 1) * max_applies);
  for (auto& e : p.ev) CK(cudaEventCreate(&e));
  p.on = true;
  return SCABEM_OK;
}

int scabem_profile_read(scabem_op_t op, double* stage_ms, int64_t* n_applies) {
  if (!op || !stage_ms) {
    set_error("scabem_profile_read: null argument");
    return SCABEM_E_ARG;
  }
  Profiler& p = op->prof;
  const int64_t n = p.used / (NSTAGE + 1);
  for (int k = 0; k < NSTAGE; ++k) stage_ms[k] = 0.0;
  for (int64_t a = 0; a < n; ++a) {
    for (int k = 0; k < NSTAGE; ++k) {
      float ms = 0.f;
      cudaEvent_t e0 = p.ev[a * (NSTAGE + 1) + k], e1 = p.ev[a * (NSTAGE + 1) + k + 1];
      CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(&ms, e0, e1));
      stage_ms[k] += ms;
    }
  }
  if (n_applies) *n_applies = n;
  p.used = 0;
  return SCABEM_OK;
}

void scabem_op_destroy(scabem_op_t op) {
  if (!op) return;
  for (auto e : op->prof.ev) cudaEventDestroy(e);
  circulant_release(op);
  cudaFree(op->tri);
  cudaFree(op->cX);
  cudaFree(op->unk);
  cudaFree(op->region);
  cudaFree(op->trirow);
  cudaFree(op->valrow);
  cudaFree(op->rowsrc);
  cudaFree(op->qp);
  cudaFree(op->qw);
  cudaFree(op->base);
  cudaFree(op->goff);
  cudaFree(op->gent);
  cudaFree(op->gpt);
  cudaFree(op->gwd);
  cudaFree(op->gwf);
  cudaFree(op->sig64);
  cudaFree(op->noff);
  cudaFree(op->nsrc);
  cudaFree(op->gspatial[0]);
  cudaFree(op->gspatial[1]);
  cudaFree(op->etk);
  cudaFree(op->ecls);
  cudaFree(op->eunk);
  cudaFree(op->pinv);
  cudaFree(op->err);
  cudaFree(op->acol);
  cudaFree(op->gdd);
  cudaFree(op->gdf);
  cudaFree(op->roff);
  cudaFree(op->rpair);
  cudaFree(op->xsrc);
  cudaFree(op->acoord);
  if (op->tmo_h) cudaFreeHost(op->tmo_h);
  free_prec(op->f);
  free_prec(op->d);
  delete op;
}

int scabem_set_sigma(scabem_op_t op, const scabem_sigma* sg) {
  if (!op || !sg) {
    set_error("scabem_set_sigma: null argument");
    return SCABEM_E_ARG;
  }
  cudaStream_t s = nullptr;
  if (sg->kind == SCABEM_SIGMA_MONOMIAL) {
    if (sg->nseg < 0 || (sg->nseg > 0 && !sg->seg)) {
      set_error("monomial profile: bad segment list");
      return SCABEM_E_ARG;
    }
    for (int i = 0; i < sg->nseg; ++i) {
      const double* g = sg->seg + 6 * i;
      for (int c = 0; c < 6; ++c)
        if (!std::isfinite(g[c])) {
          set_error("monomial profile: non-finite parameter");
          return SCABEM_E_NONFINITE;
        }
      if (!(g[1] > 0) || g[2] < 0 || g[3] < 0 || (g[4] != 0 && g[4] != 1 && g[4] != 2) ||
          (g[5] != 1 && g[5] != -1)) {
        set_error("monomial profile: need L > 0, sigma0 >= 0, d >= 0, axis in {0,1,2}, dir = +-1");
        return SCABEM_E_ARG;
      }
    }
    return setup_sigma_monomial(op, sg->nseg, sg->seg, s);
  }
  if (sg->kind == SCABEM_SIGMA_BSPLINE) {
    if (!sg->coef || sg->ncoef < 4 || sg->ncoef > 1024 || !(sg->L > 0) || sg->axis < 0 || sg->axis > 2) {
      set_error("B-spline profile: need coef, 4 <= ncoef <= 1024, L > 0, axis in {0,1,2}");
      return SCABEM_E_ARG;
    }
    if (!std::isfinite(sg->x0) || !std::isfinite(sg->L)) {
      set_error("B-spline profile: non-finite x0 or L");
      return SCABEM_E_NONFINITE;
    }
    for (int i = 0; i < sg->ncoef; ++i) {
      if (!std::isfinite(sg->coef[i])) {
        set_error("B-spline profile: non-finite coefficient");
        return SCABEM_E_NONFINITE;
      }
      if (sg->coef[i] < 0) {
        set_error("B-spline profile: negative coefficient");
        return SCABEM_E_ARG;
      }
    }
    return setup_sigma_bspline(op, sg->x0, sg->L, sg->axis, sg->ncoef, sg->coef, s);
  }
  if (sg->kind == SCABEM_SIGMA_PER_QPOINT) {
    if (!sg->per_qpoint) {
      set_error("per-point profile: null array");
      return SCABEM_E_ARG;
    }
    for (int64_t i = 0; i < op->Q; ++i) {
      if (!std::isfinite(sg->per_qpoint[i])) {
        set_error("per-point profile: non-finite conductivity");
        return SCABEM_E_NONFINITE;
      }
      if (sg->per_qpoint[i] < 0) {
        set_error("per-point profile: negative conductivity");
        return SCABEM_E_ARG;
      }
    }
    return setup_sigma_values(op, sg->per_qpoint, s);
  }
  set_error("unknown conductivity kind");
  return SCABEM_E_ARG;
}

// Reports (once) that a bounded device wait of an earlier launch expired.
static int take_timeout(scabem_op* op) {
  volatile int* f = op->tmo_h;
  if (f && *f) {
    *f = 0;
    set_error("a bounded device wait expired in an earlier launch (near-field record stream): "
              "the results of the launches since the previous call are not valid");
    return SCABEM_E_TIMEOUT;
  }
  return SCABEM_OK;
}

int scabem_selftest_wait_limit(scabem_op_t op, void* stream) {
  if (!op) {
    set_error("scabem_selftest_wait_limit: null operator");
    return SCABEM_E_ARG;
  }
  if (int rc = take_timeout(op)) return rc;
  if (int rc = selftest_wait(op, (cudaStream_t)stream)) return rc;
  return take_timeout(op);
}

int scabem_apply(scabem_op_t op, const void* x, void* y, int32_t nrhs, int64_t ld, int32_t prec, void* stream) {
  if (!op || !x || !y || nrhs < 0 || ld < op->N) {
    set_error("scabem_apply: null argument, nrhs < 0 or ld < N");
    return SCABEM_E_ARG;
  }
  if (int rc = take_timeout(op)) return rc;
  if (nrhs == 0) return SCABEM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == SCABEM_C64) return apply_prec<float>(op, x, y, nrhs, ld, s, false);
  if (prec == SCABEM_C128) return apply_prec<double>(op, x, y, nrhs, ld, s, false);
  set_error("scabem_apply: prec must be SCABEM_C64 or SCABEM_C128");
  return SCABEM_E_ARG;
}

int scabem_apply_adjoint(scabem_op_t op, const void* y, void* x, int32_t nrhs, int64_t ld, int32_t prec,
                         void* stream) {
  if (!op || !x || !y || nrhs < 0 || ld < op->N) {
    set_error("scabem_apply_adjoint: null argument, nrhs < 0 or ld < N");
    return SCABEM_E_ARG;
  }
  if (int rc = take_timeout(op)) return rc;
  if (nrhs == 0) return SCABEM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == SCABEM_C64) return apply_prec<float>(op, y, x, nrhs, ld, s, true);
  if (prec == SCABEM_C128) return apply_prec<double>(op, y, x, nrhs, ld, s, true);
  set_error("scabem_apply_adjoint: prec must be SCABEM_C64 or SCABEM_C128");
  return SCABEM_E_ARG;
}

int scabem_rhs(scabem_op_t op, const scabem_source* src, int32_t nsrc, void* b, int64_t ld, int32_t prec,
               void* stream) {
  if (!op || !src || !b || nsrc < 0 || ld < op->N || (prec != SCABEM_C64 && prec != SCABEM_C128)) {
    set_error("scabem_rhs: bad argument");
    return SCABEM_E_ARG;
  }
  for (int i = 0; i < nsrc; ++i)
    if (src[i].kind < 0 || src[i].kind > 2 || src[i].side < 0 || src[i].side > 1) {
      set_error("scabem_rhs: source kind must be 0..2 and side 0..1");
      return SCABEM_E_ARG;
    }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t es = prec == SCABEM_C64 ? sizeof(cx<float>) : sizeof(cx<double>);
  if (is_device_ptr(b)) return rhs_impl(op, src, nsrc, b, ld, prec, s);
  void* db = nullptr;
  CK(cudaMalloc(&db, es * ld * std::max(nsrc, 1)));
  int rc = rhs_impl(op, src, nsrc, db, ld, prec, s);
  if (rc == SCABEM_OK) {
    CK(cudaMemcpyAsync(b, db, es * ld * nsrc, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  cudaFree(db);
  return rc;
}

int scabem_solve(scabem_op_t op, const void* b, void* x, int32_t nrhs, int64_t ld, const scabem_solve_opts* o,
                 void* stream, scabem_solve_info* info) {
  if (!op || !b || !x || !o || nrhs < 0 || ld < op->N || o->restart < 1 || o->restart > 200 || o->maxit < 1 ||
      !(o->tol > 0) || (o->prec != SCABEM_C64 && o->prec != SCABEM_C128) || o->transpose < 0 || o->transpose > 1) {
    set_error("scabem_solve: bad argument");
    return SCABEM_E_ARG;
  }
  if (!op->d.built) {
    set_error("scabem_solve needs the complex128 operator (prec_mask bit 1) for the FP64 residual");
    return SCABEM_E_ARG;
  }
  if (o->prec == SCABEM_C64 && !op->f.built) {
    set_error("scabem_solve in complex64 mode needs the complex64 operator (prec_mask bit 0)");
    return SCABEM_E_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = take_timeout(op)) return rc;
  const bool bd = is_device_ptr(b), xd = is_device_ptr(x);
  if (bd && xd) {
    const int rc = solve_impl(op, b, x, nrhs, ld, o, s, info);
    const int rt = take_timeout(op);  // solve_impl synchronises the stream
    return rt ? rt : rc;
  }
  const size_t bytes = sizeof(cx<double>) * ld * nrhs;
  void *db = nullptr, *dx = nullptr;
  CK(cudaMalloc(&db, bytes));
  CK(cudaMalloc(&dx, bytes));
  CK(cudaMemcpyAsync(db, b, bytes, bd ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dx, x, bytes, xd ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  int rc = solve_impl(op, db, dx, nrhs, ld, o, s, info);
  CK(cudaMemcpyAsync(x, dx, bytes, xd ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  cudaFree(db);
  cudaFree(dx);
  const int rt = take_timeout(op);
  return rt ? rt : rc;
}

int scabem_sigma_gradient(scabem_op_t op, const void* x, const void* lam, const scabem_source* src, int32_t nsrc,
                          const scabem_sigma* basis, double* g_out, void* stream) {
  if (!op || !x || !lam || !basis || !g_out || nsrc < 0 || (nsrc > 0 && !src)) {
    set_error("scabem_sigma_gradient: null argument or nsrc < 0");
    return SCABEM_E_ARG;
  }
  if (!op->d.built) {
    set_error("scabem_sigma_gradient needs the complex128 operator (prec_mask bit 1)");
    return SCABEM_E_ARG;
  }
  if (basis->kind == SCABEM_SIGMA_BSPLINE) {
    if (basis->ncoef < 4 || basis->ncoef > 1024 || !(basis->L > 0) || basis->axis < 0 || basis->axis > 2 ||
        !std::isfinite(basis->x0)) {
      set_error("scabem_sigma_gradient: B-spline basis needs 4 <= ncoef <= 1024, L > 0, axis in {0,1,2}");
      return SCABEM_E_ARG;
    }
  } else if (basis->kind == SCABEM_SIGMA_MONOMIAL) {
    if (basis->nseg < 0 || (basis->nseg > 0 && !basis->seg)) {
      set_error("scabem_sigma_gradient: monomial basis needs its segments");
      return SCABEM_E_ARG;
    }
    for (int i = 0; i < basis->nseg; ++i) {
      const double* gsg = basis->seg + 6 * i;
      if (!(gsg[1] > 0) || gsg[3] < 0 || (gsg[4] != 0 && gsg[4] != 1 && gsg[4] != 2) || (gsg[5] != 1 && gsg[5] != -1)) {
        set_error("scabem_sigma_gradient: monomial segment needs L > 0, d >= 0, axis in {0,1,2}, dir = +-1");
        return SCABEM_E_ARG;
      }
    }
  } else if (basis->kind != SCABEM_SIGMA_PER_QPOINT) {
    set_error("scabem_sigma_gradient: unknown basis kind");
    return SCABEM_E_ARG;
  }
  for (int i = 0; i < nsrc; ++i)
    if (src[i].kind < 0 || src[i].kind > 2 || src[i].side < 0 || src[i].side > 1) {
      set_error("scabem_sigma_gradient: source kind must be 0..2 and side 0..1");
      return SCABEM_E_ARG;
    }
  if (int rc = take_timeout(op)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(cx<double>) * op->N;
  const bool xd = is_device_ptr(x), ld_ = is_device_ptr(lam);
  void *dx = nullptr, *dl = nullptr;
  if (!xd) {
    CK(cudaMalloc(&dx, bytes));
    CK(cudaMemcpyAsync(dx, x, bytes, cudaMemcpyHostToDevice, s));
  }
  if (!ld_) {
    CK(cudaMalloc(&dl, bytes));
    CK(cudaMemcpyAsync(dl, lam, bytes, cudaMemcpyHostToDevice, s));
  }
  int rc = sigma_gradient_impl(op, (const cx<double>*)(xd ? x : dx), (const cx<double>*)(ld_ ? lam : dl), src, nsrc,
                               basis, g_out, s);
  cudaFree(dx);
  cudaFree(dl);
  const int rt = take_timeout(op);
  return rt ? rt : rc;
}

int scabem_fields(scabem_op_t op, const void* x, int32_t nrhs, int64_t ld, const double* pts, int32_t npts,
                  const scabem_source* inc, double* E, void* stream) {
  if (!op || !x || !pts || !E || npts <= 0 || nrhs < 0 || ld < op->N) {
    set_error("scabem_fields: bad argument");
    return SCABEM_E_ARG;
  }
  if (!op->d.built) {
    set_error("scabem_fields needs the complex128 operator");
    return SCABEM_E_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (is_device_ptr(x)) return fields_impl(op, x, nrhs, ld, pts, npts, inc, E, s);
  void* dx = nullptr;
  const size_t bytes = sizeof(cx<double>) * ld * nrhs;
  CK(cudaMalloc(&dx, bytes));
  CK(cudaMemcpyAsync(dx, x, bytes, cudaMemcpyHostToDevice, s));
  int rc = fields_impl(op, dx, nrhs, ld, pts, npts, inc, E, s);
  cudaFree(dx);
  return rc;
}

}  // extern "C"

namespace {
// Reallocate the axis-0 intermediates of one precision for the current
// (y, z) mode and batch capacity (zero, as at creation).
template <typename R>
int realloc_st(scabem_op* op, PrecData<R>& pd, cudaStream_t s) {
  if (!pd.built) return SCABEM_OK;
  cudaFree(pd.stA);
  cudaFree(pd.stB);
  pd.stA = pd.stB = nullptr;
  const int64_t n = col_stride_st(op) * pd.kcap;
  int rc;
  if ((rc = dalloc(&pd.stA, n)) || (rc = dalloc(&pd.stB, n))) return rc;
  CK(cudaMemsetAsync(pd.stA, 0, sizeof(cx<R>) * n, s));
  CK(cudaMemsetAsync(pd.stB, 0, sizeof(cx<R>) * n, s));
  return SCABEM_OK;
}

int set_transverse_mode(scabem_op* op, bool direct, cudaStream_t s) {
  if (direct == op->tdirect) return SCABEM_OK;
  CK(cudaStreamSynchronize(s));
  op->tdirect = direct;
  op->cst = direct ? op->nac : (int64_t)op->n[1] * op->n[2];
  int rc = realloc_st(op, op->d, s);
  if (!rc) rc = realloc_st(op, op->f, s);
  return rc;
}

template <typename R>
__global__ void k_tune_pattern(cx<R>* x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = mk((R)sin(0.37 * (double)(i % 100003)), (R)cos(0.11 * (double)(i % 99991)));
}

template <typename R>
int autotune_prec(scabem_op* op, int nrhs, cudaStream_t s, double* out) {
  PrecData<R>& pd = *reinterpret_cast<PrecData<R>*>(sizeof(R) == 4 ? (void*)&op->f : (void*)&op->d);
  if (nrhs > 1)
    if (int rc = ensure_batch<R>(op, nrhs, s)) return rc;
  const int64_t N = op->N;
  cx<R>* x = nullptr;
  cx<R>* y = nullptr;
  if (int rc = dalloc(&x, N * nrhs)) return rc;
  if (int rc = dalloc(&y, N * nrhs)) {
    cudaFree(x);
    return rc;
  }
  k_tune_pattern<R><<<152, 256, 0, s>>>(x, N * nrhs);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = SCABEM_OK;
  auto timed = [&](float& ms) -> int {
    auto apply = [&]() { return nrhs == 1 ? apply_one<R>(op, x, y, s) : apply_batch<R>(op, x, N, y, N, nrhs, s); };
    if (int r = apply()) return r;  // warm
    CK(cudaEventRecord(e0, s));
    for (int i = 0; i < 5; ++i)
      if (int r = apply()) return r;
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    ms /= 5;
    return SCABEM_OK;
  };
  float ms0 = 0.f;
  const bool dir0 = op->tdirect;
  const int lines0 = op->a0_lines;
  do {
    if ((rc = timed(ms0))) break;
    float best = ms0;
    bool bdir = dir0;
    int blines = lines0;
    const int csz = (int)sizeof(cx<R>);
    const int totl = sizeof(R) == 4 ? 13 : 12;  // largest transform one CTA holds (log2 elements)
    int lp = 0;
    while ((1 << lp) < op->P[0]) ++lp;
    for (int mode = 0; mode < 2 && !rc; ++mode) {
      const bool direct = mode == 0;
      if (direct ? !op->direct_fits : !op->planes_fit) continue;
      if ((rc = set_transverse_mode(op, direct, s))) break;
      for (int L = 1; L <= 16 && !rc; L *= 2) {
        const int cbC = L >= 4 ? L : 4;
        if ((1 << lp) * L > (1 << totl) || (1 << lp) * cbC > (1 << totl) ||
            (int64_t)op->P[0] * (L + 1) * csz > 227 * 1024 || (int64_t)op->P[0] * (cbC + 1) * csz > 227 * 1024)
          continue;
        op->a0_lines = L;
        float ms = 0.f;
        if ((rc = timed(ms))) break;
        if (ms < best) {
          best = ms;
          bdir = direct;
          blines = L;
        }
      }
    }
    if (rc) break;
    if ((rc = set_transverse_mode(op, bdir, s))) break;
    op->a0_lines = blines;
    out[0] = best;
    out[1] = ms0;
    out[2] = bdir ? 1.0 : 0.0;
    out[3] = blines > 0 ? blines : 0.0;
  } while (0);
  if (rc) {  // leave the operator as it was
    set_transverse_mode(op, dir0, s);
    op->a0_lines = lines0;
  }
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  return rc;
}
}  // namespace

extern "C" {

int scabem_autotune(scabem_op_t op, int32_t prec, int32_t nrhs, void* stream, double* out) {
  if (!op || !out || (prec != SCABEM_C64 && prec != SCABEM_C128) || nrhs < 1 || nrhs > KBATCH) {
    set_error("scabem_autotune: bad argument (prec SCABEM_C64 or SCABEM_C128, 1 <= nrhs <= 8)");
    return SCABEM_E_ARG;
  }
  if ((prec == SCABEM_C64 && !op->f.built) || (prec == SCABEM_C128 && !op->d.built)) {
    set_error("scabem_autotune: the operator was not built for this precision");
    return SCABEM_E_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = take_timeout(op)) return rc;
  const int rc = prec == SCABEM_C64 ? autotune_prec<float>(op, nrhs, s, out) : autotune_prec<double>(op, nrhs, s, out);
  const int rt = take_timeout(op);
  return rc ? rc : rt;
}

int scabem_set_precond_circulant(scabem_op_t op, scabem_mesh_t mesh, const scabem_circulant* c, void* stream) {
  if (!op || !mesh || !c || c->axis < 0 || c->axis > 2 || !(c->dx > 0) || !std::isfinite(c->x0) || c->first < 0 ||
      c->count < 0 || (c->count > 0 && c->count < 2) || c->count > 4096 || mesh->nt != op->nt || mesh->N != op->N ||
      c->kind < 0 || c->kind > 1) {
    set_error("scabem_set_precond_circulant: bad argument (axis 0..2, dx > 0, first >= 0, count 0 or 2..4096, "
              "kind 0 or 1, the operator's mesh)");
    return SCABEM_E_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = take_timeout(op)) return rc;
  const int rc = setup_circulant(op, mesh, c, s);
  const int rt = take_timeout(op);
  return rc ? rc : rt;
}

int scabem_precond_apply(scabem_op_t op, const void* v, void* z, int32_t nrhs, int64_t ld, int32_t transpose,
                         void* stream) {
  if (!op || !v || !z || nrhs < 0 || ld < op->N || transpose < 0 || transpose > 1) {
    set_error("scabem_precond_apply: bad argument");
    return SCABEM_E_ARG;
  }
  if (nrhs == 0) return SCABEM_OK;
  if (!is_device_ptr(v) || !is_device_ptr(z)) {
    set_error("scabem_precond_apply: v and z must be device memory");
    return SCABEM_E_ARG;
  }
  return precond_apply(op, (const cx<double>*)v, (cx<double>*)z, (cudaStream_t)stream, transpose != 0, nrhs, ld, ld);
}

int scabem_fields_eh(scabem_op_t op, const void* x, int32_t nrhs, int64_t ld, const double* pts, int32_t npts,
                     int32_t side, const scabem_source* inc, double* E, double* H, void* stream) {
  if (!op || !x || !pts || !E || !H || npts <= 0 || nrhs < 0 || ld < op->N || side < 0 || side > 1) {
    set_error("scabem_fields_eh: bad argument (npts > 0, side 0 or 1, ld >= N)");
    return SCABEM_E_ARG;
  }
  if (!op->d.built) {
    set_error("scabem_fields_eh needs the complex128 operator");
    return SCABEM_E_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  return with_device_x(op, x, nrhs, ld, s, [&](const void* dx) {
    return fields_eh_impl(op, dx, nrhs, ld, pts, npts, side, inc, E, H, s);
  });
}

int scabem_poynting_rate(scabem_op_t op, const void* x, int32_t nrhs, int64_t ld, const scabem_poynting* p,
                         const scabem_source* inc, double* out, void* stream) {
  if (!op || !x || !p || !out || nrhs < 0 || ld < op->N || p->n < 1 || p->n > 64 || !(p->core[0] > 0) ||
      !(p->core[1] > 0) || !(p->box[0] > p->core[0]) || !(p->box[1] > p->core[1]) || !(p->slab > 0) ||
      !std::isfinite(p->xc)) {
    set_error("scabem_poynting_rate: bad argument (1 <= n <= 64, 0 < core < box, slab > 0)");
    return SCABEM_E_ARG;
  }
  if (!op->d.built) {
    set_error("scabem_poynting_rate needs the complex128 operator");
    return SCABEM_E_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  return with_device_x(op, x, nrhs, ld, s, [&](const void* dx) {
    return poynting_impl(op, dx, nrhs, ld, p, inc, out, s);
  });
}

static bool decay_grid_ok(double alo, double ahi, int32_t na, double blo, double bhi, int32_t nb) {
  return na >= 1 && nb >= 1 && (int64_t)na * nb <= (1 << 24) && std::isfinite(alo) && std::isfinite(ahi) &&
         std::isfinite(blo) && std::isfinite(bhi);
}

int scabem_decay_fit(const double* t, const double* E, int32_t npts, double alpha_lo, double alpha_hi,
                     int32_t nalpha, double beta_lo, double beta_hi, int32_t nbeta, double* out, void* stream) {
  if (!t || !E || !out || npts < 4 || !decay_grid_ok(alpha_lo, alpha_hi, nalpha, beta_lo, beta_hi, nbeta)) {
    set_error("scabem_decay_fit: bad argument (npts >= 4, nalpha, nbeta >= 1, nalpha * nbeta <= 2^24, finite ranges)");
    return SCABEM_E_ARG;
  }
  for (int i = 0; i < npts; ++i)
    if (!std::isfinite(t[i]) || !std::isfinite(E[2 * i]) || !std::isfinite(E[2 * i + 1])) {
      set_error("scabem_decay_fit: non-finite sample");
      return SCABEM_E_NONFINITE;
    }
  if (int rc = check_device()) return rc;
  return decay_fit_impl(t, E, npts, alpha_lo, alpha_hi, nalpha, beta_lo, beta_hi, nbeta, out, (cudaStream_t)stream);
}

int scabem_decay_rate(scabem_op_t op, const void* x, int32_t nrhs, int64_t ld, const scabem_probe* pr,
                      double alpha_lo, double alpha_hi, int32_t nalpha, const scabem_source* inc, double* out,
                      void* stream) {
  if (!op || !x || !pr || !out || pr->npts < 4 || pr->axis < 0 || pr->axis > 2 || pr->comp < 0 || pr->comp > 2 ||
      nrhs < 0 || ld < op->N || !decay_grid_ok(alpha_lo, alpha_hi, nalpha, pr->beta_lo, pr->beta_hi, pr->nbeta)) {
    set_error("scabem_decay_rate: bad argument (npts >= 4, axis/comp in 0..2, nalpha, nbeta >= 1, "
              "nalpha * nbeta <= 2^24)");
    return SCABEM_E_ARG;
  }
  if (!op->d.built) {
    set_error("scabem_decay_rate needs the complex128 operator");
    return SCABEM_E_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (is_device_ptr(x)) return decay_rate_impl(op, x, nrhs, ld, pr, alpha_lo, alpha_hi, nalpha, inc, out, s);
  void* dx = nullptr;
  const size_t bytes = sizeof(cx<double>) * ld * nrhs;
  CK(cudaMalloc(&dx, bytes));
  CK(cudaMemcpyAsync(dx, x, bytes, cudaMemcpyHostToDevice, s));
  int rc = decay_rate_impl(op, dx, nrhs, ld, pr, alpha_lo, alpha_hi, nalpha, inc, out, s);
  cudaFree(dx);
  return rc;
}

int scabem_reflection(scabem_op_t op, const void* x, int32_t nrhs, int64_t ld, const scabem_probe* pr,
                      const scabem_source* inc, double* out, void* stream) {
  if (!op || !x || !pr || !out || pr->npts < 4 || pr->nbeta < 1 || pr->axis < 0 || pr->axis > 2 || pr->comp < 0 ||
      pr->comp > 2 || nrhs < 0 || ld < op->N) {
    set_error("scabem_reflection: bad argument (npts >= 4, nbeta >= 1, axis/comp in 0..2)");
    return SCABEM_E_ARG;
  }
  if (!op->d.built) {
    set_error("scabem_reflection needs the complex128 operator");
    return SCABEM_E_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (is_device_ptr(x)) return reflection_impl(op, x, nrhs, ld, pr, inc, out, s);
  void* dx = nullptr;
  const size_t bytes = sizeof(cx<double>) * ld * nrhs;
  CK(cudaMalloc(&dx, bytes));
  CK(cudaMemcpyAsync(dx, x, bytes, cudaMemcpyHostToDevice, s));
  int rc = reflection_impl(op, dx, nrhs, ld, pr, inc, out, s);
  cudaFree(dx);
  return rc;
}

}  // extern "C"
