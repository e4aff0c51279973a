// Operator set-up on the device: triangle geometry and quadrature, grid
// stencils, the two Green's spectra, the near-pair list and the near-field
// precorrection, and the conductivity at the quadrature points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

// Symmetric triangle rules (Dunavant 1985): barycentric coordinates and
// weights summing to one; the point order is part of the interface.
__constant__ double c_bary[MAXQ][3];
__constant__ double c_w[MAXQ];

int load_rule(int q) {
  const double a6 = 0.445948490915965, b6 = 0.091576213509771;
  const double wa6 = 0.223381589678011, wb6 = 0.109951743655322;
  const double a7 = 0.059715871789770, b7 = 0.470142064105115;
  const double c7 = 0.797426985353087, d7 = 0.101286507323456;
  double B[MAXQ][3] = {};
  double W[MAXQ] = {};
  if (q == 1) {
    B[0][0] = B[0][1] = B[0][2] = 1.0 / 3.0;
    W[0] = 1.0;
  } else if (q == 3) {
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) B[i][j] = (i == j) ? 2.0 / 3.0 : 1.0 / 6.0;
      W[i] = 1.0 / 3.0;
    }
  } else if (q == 6) {
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) {
        B[i][j] = (i == j) ? 1.0 - 2.0 * a6 : a6;
        B[3 + i][j] = (i == j) ? 1.0 - 2.0 * b6 : b6;
      }
      W[i] = wa6;
      W[3 + i] = wb6;
    }
  } else if (q == 7) {
    B[0][0] = B[0][1] = B[0][2] = 1.0 / 3.0;
    W[0] = 0.225;
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) {
        B[1 + i][j] = (i == j) ? a7 : b7;
        B[4 + i][j] = (i == j) ? c7 : d7;
      }
      W[1 + i] = 0.132394152788506;
      W[4 + i] = 0.125939180544827;
    }
  } else {
    set_error("q must be 1, 3, 6 or 7");
    return SCABEM_E_ARG;
  }
  CK(cudaMemcpyToSymbol(c_bary, B, sizeof(B)));
  CK(cudaMemcpyToSymbol(c_w, W, sizeof(W)));
  return SCABEM_OK;
}

__device__ __forceinline__ void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// Lagrange basis on nodes 0..p-1 at t, and its derivative.
__device__ void lagrange(double t, int p, double* L, double* dL) {
  for (int i = 0; i < p; ++i) {
    double v = 1.0;
    for (int m = 0; m < p; ++m)
      if (m != i) v *= (t - m) / (double)(i - m);
    L[i] = v;
    double d = 0.0;
    for (int j = 0; j < p; ++j) {
      if (j == i) continue;
      double term = 1.0 / (double)(i - j);
      for (int m = 0; m < p; ++m)
        if (m != i && m != j) term *= (t - m) / (double)(i - m);
      d += term;
    }
    dL[i] = d;
  }
}

// Per triangle: vertices, centroid, unit normal, area, s_k l_k/(2A), and the
// quadrature points with their stencils.
__global__ void k_geometry(const double* __restrict__ V, const int32_t* __restrict__ T,
                           const int32_t* __restrict__ tsign, int64_t nt, int q, int p, double h, double ox,
                           double oy, double oz, int n0, int n1, int n2, double* __restrict__ tri,
                           double* __restrict__ cX, double* __restrict__ qp, double* __restrict__ qw,
                           int32_t* __restrict__ base, double* __restrict__ Ld, double* __restrict__ dLd,
                           float* __restrict__ Lf, float* __restrict__ dLf, int* err) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double v[3][3];
  for (int i = 0; i < 3; ++i)
    for (int c = 0; c < 3; ++c) v[i][c] = V[3 * (int64_t)T[3 * t + i] + c];
  double e1[3], e2[3], nr[3];
  for (int c = 0; c < 3; ++c) {
    e1[c] = v[1][c] - v[0][c];
    e2[c] = v[2][c] - v[0][c];
  }
  cross3(e1, e2, nr);
  const double nn = sqrt(nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
  const double area = 0.5 * nn;
  double* o = tri + 16 * t;
  for (int i = 0; i < 3; ++i)
    for (int c = 0; c < 3; ++c) o[3 * i + c] = v[i][c];
  for (int c = 0; c < 3; ++c) {
    o[9 + c] = (v[0][c] + v[1][c] + v[2][c]) / 3.0;
    o[12 + c] = nr[c] / nn;
  }
  o[15] = area;
  for (int k = 0; k < 3; ++k) {
    const double* a = v[(k + 1) % 3];
    const double* b = v[(k + 2) % 3];
    const double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
    const double len = sqrt(dx * dx + dy * dy + dz * dz);
    cX[3 * t + k] = tsign[3 * t + k] * len / (2.0 * area);
  }
  const double org[3] = {ox, oy, oz};
  const int nn3[3] = {n0, n1, n2};
  for (int a = 0; a < q; ++a) {
    const int64_t Qi = t * q + a;
    double r[3];
    for (int c = 0; c < 3; ++c) r[c] = c_bary[a][0] * v[0][c] + c_bary[a][1] * v[1][c] + c_bary[a][2] * v[2][c];
    for (int c = 0; c < 3; ++c) qp[3 * Qi + c] = r[c];
    qw[Qi] = c_w[a] * area;
    for (int ax = 0; ax < 3; ++ax) {
      const double u = (r[ax] - org[ax]) / h;
      const int b = (int)floor(u - 0.5 * (p - 2));
      base[3 * Qi + ax] = b;
      if (b < 0 || b + p - 1 >= nn3[ax]) atomicOr(err, 1);
      double L[MAXP], dL[MAXP];
      lagrange(u - b, p, L, dL);
      for (int i = 0; i < p; ++i) {
        Ld[(3 * Qi + ax) * p + i] = L[i];
        dLd[(3 * Qi + ax) * p + i] = dL[i] / h;
        Lf[(3 * Qi + ax) * p + i] = (float)L[i];
        dLf[(3 * Qi + ax) * p + i] = (float)(dL[i] / h);
      }
    }
  }
}

// G(d) = exp(-jk|d|h)/(4 pi |d| h) on the padded grid with circular offsets;
// zero at d = 0 and on the unused offset n of each axis.
__global__ void k_green_fill(cx<double>* G, int P0, int P1, int P2, int n0, int n1, int n2, double h, double k) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t tot = (int64_t)P0 * P1 * P2;
  if (idx >= tot) return;
  int i2 = (int)(idx % P2);
  int i1 = (int)((idx / P2) % P1);
  int i0 = (int)(idx / ((int64_t)P1 * P2));
  cx<double> g = mk(0.0, 0.0);
  if (i0 != n0 && i1 != n1 && i2 != n2) {
    double d0 = i0 < n0 ? i0 : i0 - P0;
    double d1 = i1 < n1 ? i1 : i1 - P1;
    double d2 = i2 < n2 ? i2 : i2 - P2;
    double dist = h * sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    if (dist > 0) {
      double s, c;
      sincos(k * dist, &s, &c);
      double inv = 1.0 / (4.0 * M_PI * dist);
      g = mk(c * inv, -s * inv);
    }
  }
  G[idx] = g;
}

// Octant of the (even) spectrum, scaled by 1/(P0 P1 P2).
__global__ void k_octant(const cx<double>* __restrict__ F, cx<double>* __restrict__ od, cx<float>* __restrict__ of,
                         int P0, int P1, int P2) {
  const int h0 = P0 / 2 + 1, h1 = P1 / 2 + 1, h2 = P2 / 2 + 1;
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t tot = (int64_t)h0 * h1 * h2;
  if (idx >= tot) return;
  int q2 = (int)(idx % h2);
  int q1 = (int)((idx / h2) % h1);
  int q0 = (int)(idx / ((int64_t)h1 * h2));
  const double sc = 1.0 / ((double)P0 * P1 * P2);
  cx<double> v = F[((int64_t)q0 * P1 + q1) * P2 + q2];
  v = sc * v;
  // stored [q0][q2][q1]: the plane kernels walk q1 along their lanes
  const int64_t o = ((int64_t)q0 * h2 + q2) * h1 + q1;
  if (od) od[o] = v;
  if (of) of[o] = mk((float)v.re, (float)v.im);
}

// Transverse tables of the direct (y, z) convolution: F holds the axis-0
// transform of the padded spatial table, [k0][i1][i2]; keep k0 <= P0/2 (even
// in k0) and offsets 0 <= d1 < R1, 0 <= d2 < R2 (even in d1, d2), scaled by
// 1/P0 for the unnormalised inverse axis-0 transform.
__global__ void k_transverse(const cx<double>* __restrict__ F, int P0, int P1, int P2, int R1, int R2,
                             cx<double>* __restrict__ od, cx<float>* __restrict__ of) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t tot = (int64_t)(P0 / 2 + 1) * R1 * R2;
  if (idx >= tot) return;
  const int d2 = (int)(idx % R2);
  const int d1 = (int)((idx / R2) % R1);
  const int q0 = (int)(idx / ((int64_t)R1 * R2));
  const cx<double> v = (1.0 / P0) * F[((int64_t)q0 * P1 + d1) * P2 + d2];
  if (od) od[idx] = v;
  if (of) of[idx] = mk((float)v.re, (float)v.im);
}

// ---------------------------------------------------------------- near list
__global__ void k_near_count(const double* __restrict__ tri, int64_t nt, double r2, int32_t* __restrict__ cnt) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const double cx0 = tri[16 * t + 9], cy0 = tri[16 * t + 10], cz0 = tri[16 * t + 11];
  int c = 0;
  for (int64_t s = 0; s < nt; ++s) {
    const double dx = cx0 - tri[16 * s + 9], dy = cy0 - tri[16 * s + 10], dz = cz0 - tri[16 * s + 11];
    if (dx * dx + dy * dy + dz * dz < r2) ++c;
  }
  cnt[t] = c;
}

__global__ void k_near_fill(const double* __restrict__ tri, int64_t nt, double r2, const int32_t* __restrict__ off,
                            int32_t* __restrict__ src) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const double cx0 = tri[16 * t + 9], cy0 = tri[16 * t + 10], cz0 = tri[16 * t + 11];
  int64_t o = off[t];
  for (int64_t s = 0; s < nt; ++s) {
    const double dx = cx0 - tri[16 * s + 9], dy = cy0 - tri[16 * s + 10], dz = cz0 - tri[16 * s + 11];
    if (dx * dx + dy * dy + dz * dz < r2) src[o++] = (int32_t)s;
  }
}

// ---------------------------------------------------------------- panel integrals
// Closed-form int 1/R, int (rho'-rho)/R and int grad_r(1/R) over the flat
// triangle (singularity extraction of Eqs. 15-16; line-integral formulas of
// Wilton et al. / Graglia restated from the divergence theorem).
__device__ void static_tri(const double* r, const double* v, const double* nrm, bool self, double& I,
                           double* Irho, double* gI, double* rho) {
  const double d0 = (r[0] - v[0]) * nrm[0] + (r[1] - v[1]) * nrm[1] + (r[2] - v[2]) * nrm[2];
  const double d = self ? 0.0 : d0;
  const double ad = fabs(d);
  for (int c = 0; c < 3; ++c) rho[c] = r[c] - d * nrm[c];
  I = 0.0;
  double om = 0.0;
  for (int c = 0; c < 3; ++c) Irho[c] = gI[c] = 0.0;
  for (int e = 0; e < 3; ++e) {
    const double* a = v + 3 * e;
    const double* b = v + 3 * ((e + 1) % 3);
    double lv[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const double ll = sqrt(lv[0] * lv[0] + lv[1] * lv[1] + lv[2] * lv[2]);
    for (int c = 0; c < 3; ++c) lv[c] /= ll;
    double uh[3];
    cross3(lv, nrm, uh);
    double am[3] = {a[0] - rho[0], a[1] - rho[1], a[2] - rho[2]};
    double bm[3] = {b[0] - rho[0], b[1] - rho[1], b[2] - rho[2]};
    const double sm = am[0] * lv[0] + am[1] * lv[1] + am[2] * lv[2];
    const double sp = bm[0] * lv[0] + bm[1] * lv[1] + bm[2] * lv[2];
    const double t = am[0] * uh[0] + am[1] * uh[1] + am[2] * uh[2];
    const double r0 = t * t + d * d;
    const double Rm = sqrt(r0 + sm * sm), Rp = sqrt(r0 + sp * sp);
    const double f = (sp + sm > 0) ? log((Rp + sp) / (Rm + sm)) : log((Rm - sm) / (Rp - sp));
    const double be = atan2(t * sp, r0 + ad * Rp) - atan2(t * sm, r0 + ad * Rm);
    I += t * f - ad * be;
    const double g = 0.5 * (r0 * f + sp * Rp - sm * Rm);
    for (int c = 0; c < 3; ++c) {
      Irho[c] += g * uh[c];
      gI[c] -= f * uh[c];
    }
    om += be;
  }
  const double sg = (d > 0) ? 1.0 : ((d < 0) ? -1.0 : 0.0);
  for (int c = 0; c < 3; ++c) gI[c] -= sg * om * nrm[c];
}

// Near-field precorrection: one thread per (near pair, target point).  For
// both media, exact potential moments (P0, P1, Q, C) of the source panel at
// the target point minus the grid's version of the same interaction.
// corr layout: [pair][target point][medium][NCORR component], so that the ten
// values one (point, medium) lane of the point kernel reads are contiguous.
template <typename RG>
__global__ void k_near_corr(const double* __restrict__ tri, const double* __restrict__ qp, const double* __restrict__ qw,
                            const int32_t* __restrict__ base, const double* __restrict__ Ld,
                            const double* __restrict__ dLd, const int32_t* __restrict__ noff,
                            const int32_t* __restrict__ nsrc, int64_t nt, int64_t npairs, int q, int p, double ke,
                            double ki, const cx<RG>* __restrict__ Ge, const cx<RG>* __restrict__ Gi, int P0, int P1,
                            int P2, cx<double>* __restrict__ outd, cx<float>* __restrict__ outf) {
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= npairs * q) return;
  const int64_t j = gid / q;
  const int a = (int)(gid - j * q);
  // target triangle: binary search in noff
  int64_t lo = 0, hi = nt;
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) / 2;
    if (noff[mid] <= j) lo = mid;
    else hi = mid;
  }
  const int64_t t = lo;
  const int64_t s = nsrc[j];
  const int64_t Qa = t * q + a;
  const double r[3] = {qp[3 * Qa], qp[3 * Qa + 1], qp[3 * Qa + 2]};
  const double* ts = tri + 16 * s;
  const double cs[3] = {ts[9], ts[10], ts[11]};
  const bool self = (s == t);
  double I, Irho[3], gI[3], rho[3];
  static_tri(r, ts, ts + 12, self, I, Irho, gI, rho);
  const double inv4pi = 1.0 / (4.0 * M_PI);
  // target stencil weights
  const int ba[3] = {base[3 * Qa], base[3 * Qa + 1], base[3 * Qa + 2]};
  double La[3][MAXP], dLa[3][MAXP];
  for (int ax = 0; ax < 3; ++ax)
    for (int i = 0; i < p; ++i) {
      La[ax][i] = Ld[(3 * Qa + ax) * p + i];
      dLa[ax][i] = dLd[(3 * Qa + ax) * p + i];
    }
  const int nd = 2 * p - 1;
  for (int med = 0; med < 2; ++med) {
    const double k = med == 0 ? ke : ki;
    const cx<RG>* G = med == 0 ? Ge : Gi;
    cx<double> P0s = mk(0.0, 0.0), P1s[3], Qs[3];
    cx<double> P0g = mk(0.0, 0.0), P1g[3], Qg[3], Cg[3];
    for (int c = 0; c < 3; ++c) P1s[c] = Qs[c] = P1g[c] = Qg[c] = Cg[c] = mk(0.0, 0.0);
    for (int b = 0; b < q; ++b) {
      const int64_t Qb = s * q + b;
      const double rb[3] = {qp[3 * Qb], qp[3 * Qb + 1], qp[3 * Qb + 2]};
      const double wb = qw[Qb];
      const double rel[3] = {rb[0] - cs[0], rb[1] - cs[1], rb[2] - cs[2]};
      const double D[3] = {r[0] - rb[0], r[1] - rb[1], r[2] - rb[2]};
      // smooth remainder (exp(-jkR) - 1)/R and its radial derivative
      cx<double> gv, gd;
      if (self && b == a) {
        gv = mk(0.0, -k);
        gd = mk(0.0, 0.0);
      } else {
        const double R = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
        const double kr = k * R;
        double sn, cn, sh, ch;
        sincos(kr, &sn, &cn);
        sincos(0.5 * kr, &sh, &ch);
        gv = mk(-2.0 * sh * sh / R, -sn / R);
        gd = mk((2.0 * sh * sh - kr * sn) / (R * R * R), (sn - kr * cn) / (R * R * R));
      }
      P0s += wb * gv;
      for (int c = 0; c < 3; ++c) {
        P1s[c] += (wb * rel[c]) * gv;
        Qs[c] += (wb * D[c]) * gd;
      }
      // grid interaction Gh(a,b) and grad_a Gh(a,b), separable over axes
      const int bb[3] = {base[3 * Qb], base[3 * Qb + 1], base[3 * Qb + 2]};
      double K[3][2 * MAXP - 1], dK[3][2 * MAXP - 1];
      for (int ax = 0; ax < 3; ++ax) {
        double Lb[MAXP];
        for (int i = 0; i < p; ++i) Lb[i] = Ld[(3 * Qb + ax) * p + i];
        for (int dd = 0; dd < nd; ++dd) {
          const int delta = dd - (p - 1);
          double sv = 0.0, sd = 0.0;
          for (int i = 0; i < p; ++i) {
            const int ip = i - delta;
            if (ip < 0 || ip >= p) continue;
            sv += La[ax][i] * Lb[ip];
            sd += dLa[ax][i] * Lb[ip];
          }
          K[ax][dd] = sv;
          dK[ax][dd] = sd;
        }
      }
      const int Dg[3] = {ba[0] - bb[0], ba[1] - bb[1], ba[2] - bb[2]};
      cx<double> gh = mk(0.0, 0.0), gx = gh, gy = gh, gz = gh;
      for (int dx = 0; dx < nd; ++dx) {
        int o0 = Dg[0] + dx - (p - 1);
        o0 = o0 < 0 ? o0 + P0 : o0;
        for (int dy = 0; dy < nd; ++dy) {
          int o1 = Dg[1] + dy - (p - 1);
          o1 = o1 < 0 ? o1 + P1 : o1;
          const double kxy = K[0][dx] * K[1][dy];
          const double dxy = dK[0][dx] * K[1][dy];
          const double xdy = K[0][dx] * dK[1][dy];
          const cx<RG>* row = G + ((int64_t)o0 * P1 + o1) * P2;
          for (int dz = 0; dz < nd; ++dz) {
            int o2 = Dg[2] + dz - (p - 1);
            o2 = o2 < 0 ? o2 + P2 : o2;
            const cx<RG> gg = row[o2];
            const cx<double> g = mk((double)gg.re, (double)gg.im);
            axpy(gh, kxy * K[2][dz], g);
            axpy(gx, dxy * K[2][dz], g);
            axpy(gy, xdy * K[2][dz], g);
            axpy(gz, kxy * dK[2][dz], g);
          }
        }
      }
      P0g += wb * gh;
      const cx<double> gg3[3] = {gx, gy, gz};
      for (int c = 0; c < 3; ++c) {
        P1g[c] += (wb * rel[c]) * gh;
        Qg[c] += wb * gg3[c];
      }
      // Cg += wb * grad Gh x rel
      Cg[0] += wb * (rel[2] * gg3[1] - rel[1] * gg3[2]);
      Cg[1] += wb * (rel[0] * gg3[2] - rel[2] * gg3[0]);
      Cg[2] += wb * (rel[1] * gg3[0] - rel[0] * gg3[1]);
    }
    // exact moments
    cx<double> P0e = inv4pi * (mk(I, 0.0) + P0s);
    cx<double> P1e[3], Qe[3], Ce[3];
    for (int c = 0; c < 3; ++c) {
      P1e[c] = inv4pi * (mk(Irho[c] + (rho[c] - cs[c]) * I, 0.0) + P1s[c]);
      Qe[c] = inv4pi * (mk(gI[c], 0.0) + Qs[c]);
    }
    const double rc[3] = {r[0] - cs[0], r[1] - cs[1], r[2] - cs[2]};
    Ce[0] = rc[2] * Qe[1] - rc[1] * Qe[2];
    Ce[1] = rc[0] * Qe[2] - rc[2] * Qe[0];
    Ce[2] = rc[1] * Qe[0] - rc[0] * Qe[1];
    cx<double> o[NCORR];
    o[0] = P0e - P0g;
    for (int c = 0; c < 3; ++c) {
      o[1 + c] = P1e[c] - P1g[c];
      o[4 + c] = Qe[c] - Qg[c];
      o[7 + c] = Ce[c] - Cg[c];
    }
    // [pair][point][medium][component]
    for (int c = 0; c < NCORR; ++c) {
      const int64_t dst = ((j * q + a) * 2 + med) * NCORR + c;
      if (outd) outd[dst] = o[c];
      if (outf) outf[dst] = mk((float)o[c].re, (float)o[c].im);
    }
  }
}

// Testing geometry per quadrature point Qi (point a of triangle t), formed in
// FP64 and stored in each operator precision: the offset from the centroid
// (3), the weight, the RWG test functions X_k(r) = cX_k (r - v_k) of the three
// local edges (3 x 3) and their divergences 2 cX_k.
__global__ void k_test_geometry(const double* __restrict__ tri, const double* __restrict__ cX,
                                const double* __restrict__ qp, const double* __restrict__ qw, int64_t Q, int q,
                                double* __restrict__ td, float* __restrict__ tf) {
  const int64_t Qi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (Qi >= Q) return;
  const int64_t t = Qi / q;
  const double* g = tri + 16 * t;
  double v[16];
  for (int c = 0; c < 3; ++c) v[c] = qp[3 * Qi + c] - g[9 + c];
  v[3] = qw[Qi];
  for (int k = 0; k < 3; ++k) {
    for (int c = 0; c < 3; ++c) v[4 + 3 * k + c] = cX[3 * t + k] * (qp[3 * Qi + c] - g[3 * k + c]);
    v[13 + k] = 2.0 * cX[3 * t + k];
  }
  for (int c = 0; c < 16; ++c) {
    if (td) td[16 * Qi + c] = v[c];
    if (tf) tf[16 * Qi + c] = (float)v[c];
  }
}

// ---------------------------------------------------------------- conductivity
__global__ void k_sigma_monomial(const double* __restrict__ qp, int64_t Q, int nseg, const double* __restrict__ seg,
                                 double* __restrict__ sd, float* __restrict__ sf, double* __restrict__ s64) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Q) return;
  double sig = 0.0;
  for (int g = 0; g < nseg; ++g) {
    const double* sgp = seg + 6 * g;
    const int ax = (int)sgp[4];
    const double s = sgp[5] * (qp[3 * i + ax] - sgp[0]) / sgp[1];
    if (s < 0.0) continue;
    const double u = s > 1.0 ? 1.0 : s;
    sig += sgp[2] * pow(u, sgp[3]);
  }
  sig *= ETA0;
  s64[i] = sig;
  if (sd) sd[i] = sig;
  if (sf) sf[i] = (float)sig;
}

// Cubic B-spline profile sum_k coef[k] N_k(s), s = (x_axis - x0) / L, on the
// clamped uniform knots of ncoef coefficients over [0, 1] (interior knots
// j / (ncoef - 3)), zero outside [0, 1]: the knot span of s and de Boor's
// triangular scheme over the four coefficients that act there.
__global__ void k_sigma_bspline(const double* __restrict__ qp, int64_t Q, double x0, double L, int axis, int ncoef,
                                const double* __restrict__ coef, double* __restrict__ sd, float* __restrict__ sf,
                                double* __restrict__ s64) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Q) return;
  const double s = (qp[3 * i + axis] - x0) / L;
  double sig = 0.0;
  if (s >= 0.0 && s <= 1.0) {
    const int nspan = ncoef - 3;  // knot intervals of [0, 1]
    int j = (int)(s * nspan);     // interval [j, j+1) / nspan; s = 1 joins the last
    if (j >= nspan) j = nspan - 1;
    // knot u(m) of the clamped vector, m = 0 .. ncoef + 3
    auto knot = [&](int m) {
      const int v = m - 3;
      return v <= 0 ? 0.0 : (v >= nspan ? 1.0 : (double)v / nspan);
    };
    // span index in the full knot vector: knots[j + 3] <= s < knots[j + 4]
    const int sp = j + 3;
    double d[4];
    for (int r = 0; r < 4; ++r) d[r] = coef[sp - 3 + r];
    for (int lvl = 1; lvl <= 3; ++lvl)
      for (int r = 3; r >= lvl; --r) {
        const int m = sp - 3 + r;
        const double den = knot(m + 4 - lvl) - knot(m);
        const double al = den > 0.0 ? (s - knot(m)) / den : 0.0;
        d[r] = (1.0 - al) * d[r - 1] + al * d[r];
      }
    sig = d[3];
  }
  sig *= ETA0;
  s64[i] = sig;
  if (sd) sd[i] = sig;
  if (sf) sf[i] = (float)sig;
}

__global__ void k_sigma_copy(const double* __restrict__ in, int64_t Q, double* __restrict__ sd, float* __restrict__ sf,
                             double* __restrict__ s64) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Q) return;
  const double sig = in[i] * ETA0;
  s64[i] = sig;
  if (sd) sd[i] = sig;
  if (sf) sf[i] = (float)sig;
}

// Stencil weight W_slot(point) = Lx[i] Ly[j] Lz[k] of every projection entry
// and its derivative weights (dLx Ly Lz, Lx dLy Lz, Lx Ly dLz: the
// transposed interpolation of gradients and curls); the entry code
// (point * p^3 + slot) is then replaced by the point index.
__global__ void k_gather_weights(int32_t* __restrict__ gent, const double* __restrict__ L,
                                 const double* __restrict__ dL, int64_t ne, int p, double* __restrict__ wd,
                                 float* __restrict__ wf, double* __restrict__ gdd, float* __restrict__ gdf) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int p2 = p * p, p3 = p2 * p;
  const int code = gent[e];
  const int64_t Qi = code / p3;
  const int sl = code - (int)Qi * p3;
  const int i = sl / p2, j = (sl - i * p2) / p, k = sl - i * p2 - j * p;
  const double lx = L[(3 * Qi + 0) * p + i], ly = L[(3 * Qi + 1) * p + j], lz = L[(3 * Qi + 2) * p + k];
  const double W = lx * ly * lz;
  wd[e] = W;
  wf[e] = (float)W;
  const double D[3] = {dL[(3 * Qi + 0) * p + i] * ly * lz, lx * dL[(3 * Qi + 1) * p + j] * lz,
                       lx * ly * dL[(3 * Qi + 2) * p + k]};
  for (int c = 0; c < 3; ++c) {
    gdd[3 * e + c] = D[c];
    gdf[3 * e + c] = (float)D[c];
  }
  gent[e] = (int32_t)Qi;
}

// ---------------------------------------------------------------- block-diagonal preconditioner
using cd = cx<double>;

// Exact moments P0, P1 (about the source centroid), Q, C = Q x (r - c) of
// source triangle s at point r for wavenumber k, given the static integrals.
__device__ void exact_moments(const double* r, const double* ts, const double* __restrict__ qp,
                              const double* __restrict__ qw, int64_t s, int q, bool self, int aself, double k,
                              double I, const double* Irho, const double* gI, const double* rho, cd* o) {
  const double cs[3] = {ts[9], ts[10], ts[11]};
  cd P0s = mk(0.0, 0.0), P1s[3], Qs[3];
  for (int c = 0; c < 3; ++c) P1s[c] = Qs[c] = mk(0.0, 0.0);
  for (int b = 0; b < q; ++b) {
    const int64_t Qb = s * q + b;
    const double D[3] = {r[0] - qp[3 * Qb], r[1] - qp[3 * Qb + 1], r[2] - qp[3 * Qb + 2]};
    const double wb = qw[Qb];
    cd gv, gd;
    if (self && b == aself) {
      gv = mk(0.0, -k);
      gd = mk(0.0, 0.0);
    } else {
      const double R = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
      const double kr = k * R;
      double sn, cn, sh, ch;
      sincos(kr, &sn, &cn);
      sincos(0.5 * kr, &sh, &ch);
      gv = mk(-2.0 * sh * sh / R, -sn / R);
      gd = mk((2.0 * sh * sh - kr * sn) / (R * R * R), (sn - kr * cn) / (R * R * R));
    }
    P0s += wb * gv;
    for (int c = 0; c < 3; ++c) {
      P1s[c] += (wb * (qp[3 * Qb + c] - cs[c])) * gv;
      Qs[c] += (wb * D[c]) * gd;
    }
  }
  const double f = 1.0 / (4.0 * M_PI);
  o[0] = f * (mk(I, 0.0) + P0s);
  for (int c = 0; c < 3; ++c) {
    o[1 + c] = f * (mk(Irho[c] + (rho[c] - cs[c]) * I, 0.0) + P1s[c]);
    o[4 + c] = f * (mk(gI[c], 0.0) + Qs[c]);
  }
  const double rc[3] = {r[0] - cs[0], r[1] - cs[1], r[2] - cs[2]};
  o[7] = rc[2] * o[5] - rc[1] * o[6];
  o[8] = rc[0] * o[6] - rc[2] * o[4];
  o[9] = rc[1] * o[4] - rc[0] * o[5];
}

// Potentials A, phi, grad phi, curl A of the summary (alpha, beta) from moments.
__device__ void unit_pot(const cd* m, double al, const double* be, cd* U) {
  for (int c = 0; c < 3; ++c) {
    U[c] = al * m[1 + c] - be[c] * m[0];
    U[4 + c] = (2.0 * al) * m[4 + c];
  }
  U[3] = (2.0 * al) * m[0];
  U[7] = al * m[7] - (be[2] * m[5] - be[1] * m[6]);
  U[8] = al * m[8] - (be[0] * m[6] - be[2] * m[4]);
  U[9] = al * m[9] - (be[1] * m[4] - be[0] * m[5]);
}

// Row values (types 0..3) at one point from J- and M-type potentials of both
// media (same expressions as the operator's testing).
__device__ void test_point(const cd* Je, const cd* Me, const cd* Ji, const cd* Mi, double ke, double ki, double ze,
                           double zi, const double* X, const double* nX, double divX, const double* n, double sg,
                           const double* Js, const double* M, cd* out) {
  const cd* J[2] = {Je, Ji};
  const cd* Mm[2] = {Me, Mi};
  const double kl[2] = {ke, ki}, zl[2] = {ze, zi};
  cd WE = mk(0.0, 0.0), WH = WE, wE = WE, wH = WE, XE[2] = {WE, WE}, nXE = WE;
  for (int m = 0; m < 2; ++m) {
    const double k = kl[m], z = zl[m], sgm = m == 0 ? 1.0 : -1.0;
    const cd* a = J[m];
    const cd* f = Mm[m];
    wE += (sgm * z / k) * mulj(a[3]);
    wH += (sgm / (k * z)) * mulj(f[3]);
    for (int c = 0; c < 3; ++c) {
      const cd we = (-z * k) * mulj(a[c]) - f[7 + c];
      const cd wh = a[7 + c] - (k / z) * mulj(f[c]);
      const cd E = -z * (k * mulj(a[c]) + (1.0 / k) * mulj(a[4 + c])) - f[7 + c];
      WE += (sgm * X[c]) * we;
      WH += (sgm * X[c]) * wh;
      XE[m] += X[c] * E;
      if (m == 0) nXE += nX[c] * E;
    }
  }
  const double nJ[3] = {n[1] * Js[2] - n[2] * Js[1], n[2] * Js[0] - n[0] * Js[2], n[0] * Js[1] - n[1] * Js[0]};
  const double nM[3] = {n[1] * M[2] - n[2] * M[1], n[2] * M[0] - n[0] * M[2], n[0] * M[1] - n[1] * M[0]};
  const double XJ = X[0] * Js[0] + X[1] * Js[1] + X[2] * Js[2];
  const double XnJ = X[0] * nJ[0] + X[1] * nJ[1] + X[2] * nJ[2];
  const double XM = X[0] * M[0] + X[1] * M[1] + X[2] * M[2];
  const double XnM = X[0] * nM[0] + X[1] * nM[1] + X[2] * nM[2];
  const cd h = WH + divX * wH;
  out[0] = WE + divX * wE;
  out[1] = h;
  out[2] = h - sg * nXE + mk(-0.5 * XnJ - 0.5 * sg * XM, 0.0);
  out[3] = mk(XJ - 0.5 * sg * XnM, 0.0) - sg * XE[1];
}

// Invert a complex n x n matrix (n <= 3) in place by Gauss-Jordan with
// partial pivoting; returns false if singular.
__device__ bool cinv(cd* A, int n) {
  cd B[9];
  for (int i = 0; i < 9; ++i) B[i] = mk(0.0, 0.0);
  for (int i = 0; i < n; ++i) B[i * 3 + i] = mk(1.0, 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    double best = 0.0;
    for (int r = c; r < n; ++r) {
      const double m = A[r * 3 + c].re * A[r * 3 + c].re + A[r * 3 + c].im * A[r * 3 + c].im;
      if (m > best) {
        best = m;
        piv = r;
      }
    }
    if (!(best > 0.0)) return false;
    if (piv != c)
      for (int j = 0; j < 3; ++j) {
        cd t = A[c * 3 + j];
        A[c * 3 + j] = A[piv * 3 + j];
        A[piv * 3 + j] = t;
        t = B[c * 3 + j];
        B[c * 3 + j] = B[piv * 3 + j];
        B[piv * 3 + j] = t;
      }
    const cd p = A[c * 3 + c];
    const double pd = p.re * p.re + p.im * p.im;
    const cd ip = mk(p.re / pd, -p.im / pd);
    for (int j = 0; j < 3; ++j) {
      A[c * 3 + j] = A[c * 3 + j] * ip;
      B[c * 3 + j] = B[c * 3 + j] * ip;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const cd fct = A[r * 3 + c];
      for (int j = 0; j < 3; ++j) {
        A[r * 3 + j] -= fct * A[c * 3 + j];
        B[r * 3 + j] -= fct * B[c * 3 + j];
      }
    }
  }
  for (int i = 0; i < 9; ++i) A[i] = B[i];
  return true;
}

// One thread per edge: the edge's own block of the operator (its two
// triangles as targets and sources, exact panel interactions), inverted.
// Columns: plain edge (J^L, M^L), absorber edge (J_e^R, J_i^R, M^R); rows:
// plain (Eq. 1, Eq. 2), absorber (Eq. 3, Eq. 13, Eq. 14).
__global__ void k_precond(const double* __restrict__ tri, const double* __restrict__ cX, const double* __restrict__ qp,
                          const double* __restrict__ qw, const double* __restrict__ sig,
                          const int32_t* __restrict__ etk, const int32_t* __restrict__ ecls, int64_t ne, int q,
                          double ke, double ki, double ze, double zi, cd* __restrict__ pinv, int* __restrict__ bad) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ne) return;
  // B[col type (Je, Ji, M)][row type 0..3]
  cd B[3][4];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 4; ++j) B[i][j] = mk(0.0, 0.0);
  const cd zero10[10] = {};
  for (int it = 0; it < 2; ++it) {
    const int64_t t = etk[4 * e + 2 * it];
    const int kt = etk[4 * e + 2 * it + 1];
    const double* gt = tri + 16 * t;
    const double cxt = cX[3 * t + kt];
    const double* n = gt + 12;
    for (int is = 0; is < 2; ++is) {
      const int64_t s = etk[4 * e + 2 * is];
      const int ks = etk[4 * e + 2 * is + 1];
      const double* gs = tri + 16 * s;
      const double al = cX[3 * s + ks];
      const double be[3] = {al * (gs[3 * ks] - gs[9]), al * (gs[3 * ks + 1] - gs[10]), al * (gs[3 * ks + 2] - gs[11])};
      const bool self = (s == t);
      for (int a = 0; a < q; ++a) {
        const int64_t Qa = t * q + a;
        const double r[3] = {qp[3 * Qa], qp[3 * Qa + 1], qp[3 * Qa + 2]};
        double I, Irho[3], gI[3], rho[3];
        static_tri(r, gs, gs + 12, self, I, Irho, gI, rho);
        cd me[10], mi[10], Ue[10], Ui[10], nUi[10];
        exact_moments(r, gs, qp, qw, s, q, self, a, ke, I, Irho, gI, rho, me);
        exact_moments(r, gs, qp, qw, s, q, self, a, ki, I, Irho, gI, rho, mi);
        unit_pot(me, al, be, Ue);
        unit_pot(mi, al, be, Ui);
        for (int c = 0; c < 10; ++c) nUi[c] = -Ui[c];
        double X[3], nX[3], Xe[3] = {0, 0, 0};
        for (int c = 0; c < 3; ++c) X[c] = cxt * (r[c] - gt[3 * kt + c]);
        nX[0] = n[1] * X[2] - n[2] * X[1];
        nX[1] = n[2] * X[0] - n[0] * X[2];
        nX[2] = n[0] * X[1] - n[1] * X[0];
        if (self)
          for (int c = 0; c < 3; ++c) Xe[c] = al * (r[c] - gs[3 * ks + c]);  // the basis itself at the point
        const double zero3[3] = {0, 0, 0};
        const double w = qw[Qa], sg = sig[Qa];
        cd o[4];
        test_point(Ue, zero10, zero10, zero10, ke, ki, ze, zi, X, nX, 2.0 * cxt, n, sg, Xe, zero3, o);
        for (int j = 0; j < 4; ++j) B[0][j] += w * o[j];
        test_point(zero10, zero10, Ui, zero10, ke, ki, ze, zi, X, nX, 2.0 * cxt, n, sg, Xe, zero3, o);
        for (int j = 0; j < 4; ++j) B[1][j] += w * o[j];
        test_point(zero10, Ue, zero10, nUi, ke, ki, ze, zi, X, nX, 2.0 * cxt, n, sg, zero3, Xe, o);
        for (int j = 0; j < 4; ++j) B[2][j] += w * o[j];
      }
    }
  }
  cd A[9];
  for (int i = 0; i < 9; ++i) A[i] = mk(0.0, 0.0);
  int nb;
  if (ecls[e] == 0) {  // rows (0, 1), cols (J = Je - Ji, M)
    nb = 2;
    for (int r = 0; r < 2; ++r) {
      A[r * 3 + 0] = B[0][r] - B[1][r];
      A[r * 3 + 1] = B[2][r];
    }
  } else {  // rows (0, 2, 3), cols (Je, Ji, M)
    nb = 3;
    const int rt[3] = {0, 2, 3};
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) A[r * 3 + c] = B[c][rt[r]];
  }
  if (!cinv(A, nb)) {
    atomicAdd(bad, 1);
    for (int i = 0; i < 9; ++i) A[i] = mk(0.0, 0.0);
    for (int i = 0; i < nb; ++i) A[i * 3 + i] = mk(1.0, 0.0);
  }
  for (int i = 0; i < 9; ++i) pinv[9 * e + i] = A[i];
}

// out[unknowns of e] = Binv_e * in[rows of e] (rows and unknowns of an edge
// share the same index set).
// transposed = 1 applies (Binv_e)^T, the inverse blocks of A^T.
__device__ __forceinline__ cd ld_cd(const cd* p) { return *p; }
__device__ __forceinline__ cd ld_cd(const cdf* p) { return df_join(*p); }

// out = P^-1 in per edge block (P^-T when transposed), read from TI
// (complex128, or FP32 (hi, lo) pairs) and written in the output precision
// TO (complex64 when it feeds the complex64 operator directly)
template <typename TI, typename TO>
__global__ void k_precond_apply(const cd* __restrict__ pinv, const int32_t* __restrict__ eunk, int64_t ne,
                                const TI* __restrict__ in, cx<TO>* __restrict__ out, int transposed, int64_t cs_in,
                                int64_t cs_out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ne) return;
  in += blockIdx.y * cs_in;  // right-hand side blockIdx.y
  out += blockIdx.y * cs_out;
  const int nb = eunk[3 * e + 2] < 0 ? 2 : 3;
  cd v[3];
  for (int i = 0; i < nb; ++i) v[i] = ld_cd(in + eunk[3 * e + i]);
  for (int i = 0; i < nb; ++i) {
    cd acc = mk(0.0, 0.0);
    for (int j = 0; j < nb; ++j) acc += pinv[9 * e + (transposed ? 3 * j + i : 3 * i + j)] * v[j];
    out[eunk[3 * e + i]] = cvt<TO>(acc);
  }
}

}  // namespace

// Inverse of the projection stencil map: for every grid point, the list of
// (quadrature point, stencil slot) pairs whose stencil covers it, in point
// order (a counting sort on the host over the device-computed stencil bases).
int setup_gather(scabem_op* op, cudaStream_t s) {
  const int p = op->p, p3 = p * p * p;
  const int64_t Q = op->Q;
  const int64_t ng = (int64_t)op->n[0] * op->n[1] * op->n[2];
  if (Q * p3 >= INT32_MAX || ng >= INT32_MAX) {
    set_error("mesh too large for the projection map");
    return SCABEM_E_ARG;
  }
  std::vector<int32_t> base(3 * Q);
  CK(cudaMemcpyAsync(base.data(), op->base, sizeof(int32_t) * 3 * Q, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int n1 = op->n[1], n2 = op->n[2];
  std::vector<int32_t> off(ng + 1, 0), ent(Q * p3);
  auto grid_index = [&](int64_t qi, int sl) {
    const int i = sl / (p * p), j = (sl / p) % p, k = sl % p;
    return ((int64_t)(base[3 * qi] + i) * n1 + (base[3 * qi + 1] + j)) * n2 + (base[3 * qi + 2] + k);
  };
  for (int64_t qi = 0; qi < Q; ++qi)
    for (int sl = 0; sl < p3; ++sl) ++off[grid_index(qi, sl) + 1];
  for (int64_t g = 0; g < ng; ++g) off[g + 1] += off[g];
  std::vector<int32_t> cur(off.begin(), off.end() - 1);
  for (int64_t qi = 0; qi < Q; ++qi)
    for (int sl = 0; sl < p3; ++sl) ent[cur[grid_index(qi, sl)]++] = (int32_t)(qi * p3 + sl);
  // compact to the grid points that some stencil covers
  std::vector<int32_t> pts, coff;
  coff.push_back(0);
  for (int64_t g = 0; g < ng; ++g)
    if (off[g + 1] > off[g]) {
      pts.push_back((int32_t)g);
      coff.push_back(off[g + 1]);
    }
  op->ngnz = (int64_t)pts.size();
  // active columns and rows of the (i1, i2) cross-section
  const int64_t C = (int64_t)n1 * n2;
  std::vector<char> colact(C, 0);
  for (int32_t g : pts) colact[g % C] = 1;
  std::vector<int32_t> acol;
  op->rowmask = 0;
  for (int64_t c = 0; c < C; ++c)
    if (colact[c]) {
      acol.push_back((int32_t)c);
      if (c / n2 < 64) op->rowmask |= 1ull << (c / n2);  // read only by the 64 x 64 plane kernel
    }
  op->nac = (int64_t)acol.size();
  if (op->nac > 0) {
    CK(cudaMalloc(&op->acol, sizeof(int32_t) * op->nac));
    CK(cudaMemcpyAsync(op->acol, acol.data(), sizeof(int32_t) * op->nac, cudaMemcpyHostToDevice, s));
    // bounding box of the active columns and their coordinates in it
    int lo1 = n1, hi1 = -1, lo2 = n2, hi2 = -1;
    for (int32_t c : acol) {
      const int i1 = c / n2, i2 = c % n2;
      lo1 = std::min(lo1, i1);
      hi1 = std::max(hi1, i1);
      lo2 = std::min(lo2, i2);
      hi2 = std::max(hi2, i2);
    }
    op->R1 = hi1 - lo1 + 1;
    op->R2 = hi2 - lo2 + 1;
    std::vector<int32_t> coord(op->nac);
    for (int64_t j = 0; j < op->nac; ++j) coord[j] = ((acol[j] / n2 - lo1) << 16) | (acol[j] % n2 - lo2);
    CK(cudaMalloc(&op->acoord, sizeof(int32_t) * op->nac));
    CK(cudaMemcpyAsync(op->acoord, coord.data(), sizeof(int32_t) * op->nac, cudaMemcpyHostToDevice, s));
  }
  {
    // one CTA of the direct (y, z) sums holds the active columns' sources and the table
    const size_t csz = (op->prec_mask & 2) ? sizeof(cx<double>) : sizeof(cx<float>);
    const size_t sm = ((size_t)op->nac * 8 + (size_t)op->R1 * op->R2) * csz + sizeof(int32_t) * op->nac;
    op->direct_fits = sm <= 227 * 1024;
    const bool want = op->transverse == 2 || !op->planes_fit ||
                      (op->transverse == 0 && op->nac * op->nac <= 16 * (int64_t)op->P[1] * op->P[2]);
    op->tdirect = want && (op->direct_fits || !op->planes_fit);
    if (op->tdirect && !op->direct_fits) {
      set_error("grid: " + std::to_string(op->nac) + " active (y, z) columns are too many for the direct sums (" +
                std::to_string(sm) + " bytes of shared memory)");
      return SCABEM_E_ARG;
    }
    if (op->transverse == 2 && !op->direct_fits) {
      set_error("grid: the direct (y, z) sums were asked for, but their columns do not fit in shared memory");
      return SCABEM_E_ARG;
    }
  }
  const int64_t ne = Q * p3;
  CK(cudaMalloc(&op->gpt, sizeof(int32_t) * (pts.size() + 1)));
  CK(cudaMalloc(&op->goff, sizeof(int32_t) * coff.size()));
  CK(cudaMalloc(&op->gent, sizeof(int32_t) * ne));
  CK(cudaMalloc(&op->gwd, sizeof(double) * ne));
  CK(cudaMalloc(&op->gwf, sizeof(float) * ne));
  CK(cudaMalloc(&op->gdd, sizeof(double) * 3 * ne));
  CK(cudaMalloc(&op->gdf, sizeof(float) * 3 * ne));
  CK(cudaMemcpyAsync(op->gpt, pts.data(), sizeof(int32_t) * pts.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(op->goff, coff.data(), sizeof(int32_t) * coff.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(op->gent, ent.data(), sizeof(int32_t) * ne, cudaMemcpyHostToDevice, s));
  k_gather_weights<<<(int)cdiv(ne, 256), 256, 0, s>>>(op->gent, op->d.L, op->d.dL, ne, p, op->gwd, op->gwf,
                                                      op->gdd, op->gdf);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return SCABEM_OK;
}

int setup_precond(scabem_op* op, cudaStream_t s) {
  CK(cudaMemsetAsync(op->err, 0, sizeof(int), s));
  k_precond<<<(int)cdiv(op->ne, 64), 64, 0, s>>>(op->tri, op->cX, op->qp, op->qw, op->sig64, op->etk, op->ecls,
                                                  op->ne, op->q, op->ke, op->ki, op->ze, op->zi, op->pinv, op->err);
  CK(cudaGetLastError());
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, op->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  op->precond_singular = bad;
  return SCABEM_OK;
}

int precond_apply(scabem_op* op, const cx<double>* in, cx<double>* out, cudaStream_t s, bool transposed, int k,
                  int64_t cs_in, int64_t cs_out) {
  k_precond_apply<cd, double><<<dim3((unsigned)cdiv(op->ne, 256), k), 256, 0, s>>>(
      op->pinv, op->eunk, op->ne, in, out, transposed ? 1 : 0, cs_in, cs_out);
  CK(cudaGetLastError());
  // the periodic plain-surface unknowns: the circulant preconditioner (forward solves)
  if (op->circ.R > 0 && !transposed) return circulant_apply(op, in, out, k, cs_in, cs_out, s);
  return SCABEM_OK;
}

bool precond_is_block_diagonal(const scabem_op* op, bool transposed) { return !(op->circ.R > 0 && !transposed); }

int precond_apply_df(scabem_op* op, const cdf* in, cx<float>* outf, cx<double>* outd, cudaStream_t s,
                     bool transposed, int k, int64_t cs_in, int64_t cs_out) {
  if (!precond_is_block_diagonal(op, transposed)) {
    set_error("internal: basis preconditioner call with a circulant block");
    return SCABEM_E_ARG;
  }
  const dim3 g((unsigned)cdiv(op->ne, 256), k);
  if (outf)
    k_precond_apply<cdf, float><<<g, 256, 0, s>>>(op->pinv, op->eunk, op->ne, in, outf, transposed ? 1 : 0, cs_in,
                                                  cs_out);
  else
    k_precond_apply<cdf, double><<<g, 256, 0, s>>>(op->pinv, op->eunk, op->ne, in, outd, transposed ? 1 : 0, cs_in,
                                                   cs_out);
  CK(cudaGetLastError());
  return SCABEM_OK;
}

int setup_geometry(scabem_op* op, const scabem_mesh* m, cudaStream_t s) {
  int rc = load_rule(op->q);
  if (rc) return rc;
  double* dV = nullptr;
  int32_t* dT = nullptr;
  int32_t* dS = nullptr;
  CK(cudaMalloc(&dV, sizeof(double) * 3 * m->nv));
  CK(cudaMalloc(&dT, sizeof(int32_t) * 3 * m->nt));
  CK(cudaMalloc(&dS, sizeof(int32_t) * 3 * m->nt));
  CK(cudaMemcpyAsync(dV, m->V.data(), sizeof(double) * 3 * m->nv, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dT, m->T.data(), sizeof(int32_t) * 3 * m->nt, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dS, m->tri_sign.data(), sizeof(int32_t) * 3 * m->nt, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(op->err, 0, sizeof(int), s));
  k_geometry<<<(int)cdiv(op->nt, 128), 128, 0, s>>>(dV, dT, dS, op->nt, op->q, op->p, op->h, op->origin[0],
                                                     op->origin[1], op->origin[2], op->n[0], op->n[1], op->n[2],
                                                     op->tri, op->cX, op->qp, op->qw, op->base, op->d.L, op->d.dL,
                                                     op->f.L, op->f.dL, op->err);
  CK(cudaGetLastError());
  k_test_geometry<<<(int)cdiv(op->Q, 256), 256, 0, s>>>(op->tri, op->cX, op->qp, op->qw, op->Q, op->q, op->d.tp,
                                                        op->f.tp);
  CK(cudaGetLastError());
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, op->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  cudaFree(dV);
  cudaFree(dT);
  cudaFree(dS);
  if (herr) {
    set_error("a quadrature point's stencil falls outside the physical grid (enlarge n or h, or move origin)");
    return SCABEM_E_ARG;
  }
  return SCABEM_OK;
}

int setup_green(scabem_op* op, cudaStream_t s) {
  const int64_t tot = (int64_t)op->P[0] * op->P[1] * op->P[2];
  const int64_t oct = (int64_t)(op->P[0] / 2 + 1) * (op->P[1] / 2 + 1) * (op->P[2] / 2 + 1);
  cx<double>* twd[3] = {nullptr, nullptr, nullptr};
  for (int a = 0; a < 3; ++a) {
    CK(cudaMalloc(&twd[a], sizeof(cx<double>) * op->P[a]));
    int rc = make_twiddles<double>(twd[a], op->P[a], s);
    if (rc) return rc;
  }
  cx<double>* F = nullptr;
  CK(cudaMalloc(&F, sizeof(cx<double>) * tot));
  for (int med = 0; med < 2; ++med) {
    const double k = med == 0 ? op->ke : op->ki;
    // spatial table kept for the near-field set-up
    CK(cudaMalloc(&op->gspatial[med], sizeof(cx<double>) * tot));
    k_green_fill<<<(int)cdiv(tot, 256), 256, 0, s>>>(op->gspatial[med], op->P[0], op->P[1], op->P[2], op->n[0],
                                                     op->n[1], op->n[2], op->h, k);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(F, op->gspatial[med], sizeof(cx<double>) * tot, cudaMemcpyDeviceToDevice, s));
    // the axis-0 transform serves both (y, z) modes: the direct sums take the
    // active box of offsets from it; the FFT planes transform on along y and z
    int rc = fft_axis_full<double>(op, F, 0, twd[0], -1, s);
    if (rc) return rc;
    if (op->direct_fits) {
      const int64_t nt_ = (int64_t)(op->P[0] / 2 + 1) * op->R1 * op->R2;
      if (op->prec_mask & 2) CK(cudaMalloc(&op->d.gt[med], sizeof(cx<double>) * nt_));
      if (op->prec_mask & 1) CK(cudaMalloc(&op->f.gt[med], sizeof(cx<float>) * nt_));
      k_transverse<<<(int)cdiv(nt_, 256), 256, 0, s>>>(F, op->P[0], op->P[1], op->P[2], op->R1, op->R2,
                                                       op->d.gt[med], op->f.gt[med]);
      CK(cudaGetLastError());
    }
    if (!op->planes_fit) continue;
    for (int a = 1; a < 3; ++a)
      if ((rc = fft_axis_full<double>(op, F, a, twd[a], -1, s))) return rc;
    if (op->prec_mask & 2) CK(cudaMalloc(&op->d.ghat[med], sizeof(cx<double>) * oct));
    if (op->prec_mask & 1) CK(cudaMalloc(&op->f.ghat[med], sizeof(cx<float>) * oct));
    k_octant<<<(int)cdiv(oct, 256), 256, 0, s>>>(F, op->d.ghat[med], op->f.ghat[med], op->P[0], op->P[1], op->P[2]);
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(s));
  cudaFree(F);
  for (int a = 0; a < 3; ++a) cudaFree(twd[a]);
  return SCABEM_OK;
}

int setup_near(scabem_op* op, cudaStream_t s) {
  const int64_t nt = op->nt;
  int32_t* cnt = nullptr;
  CK(cudaMalloc(&cnt, sizeof(int32_t) * nt));
  const double r2 = op->r_near * op->r_near;
  k_near_count<<<(int)cdiv(nt, 128), 128, 0, s>>>(op->tri, nt, r2, cnt);
  CK(cudaGetLastError());
  std::vector<int32_t> hc(nt), ho(nt + 1);
  CK(cudaMemcpyAsync(hc.data(), cnt, sizeof(int32_t) * nt, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int64_t acc = 0;
  for (int64_t t = 0; t < nt; ++t) {
    ho[t] = (int32_t)acc;
    acc += hc[t];
  }
  ho[nt] = (int32_t)acc;
  if (acc > INT32_MAX / 16) {
    set_error("near list too long: reduce r_near");
    cudaFree(cnt);
    return SCABEM_E_ARG;
  }
  op->npairs = acc;
  CK(cudaMalloc(&op->noff, sizeof(int32_t) * (nt + 1)));
  CK(cudaMalloc(&op->nsrc, sizeof(int32_t) * (acc > 0 ? acc : 1)));
  CK(cudaMemcpyAsync(op->noff, ho.data(), sizeof(int32_t) * (nt + 1), cudaMemcpyHostToDevice, s));
  k_near_fill<<<(int)cdiv(nt, 128), 128, 0, s>>>(op->tri, nt, r2, op->noff, op->nsrc);
  CK(cudaGetLastError());
  const int64_t nrec = acc * op->q * 2 * NCORR;
  if (op->prec_mask & 2) {
    cudaError_t e = cudaMalloc(&op->d.near, sizeof(cx<double>) * (nrec > 0 ? nrec : 1));
    if (e != cudaSuccess) {
      set_error("out of device memory for the near-field data");
      return SCABEM_E_NOMEM;
    }
  }
  if (op->prec_mask & 1) {
    cudaError_t e = cudaMalloc(&op->f.near, sizeof(cx<float>) * (nrec > 0 ? nrec : 1));
    if (e != cudaSuccess) {
      set_error("out of device memory for the near-field data");
      return SCABEM_E_NOMEM;
    }
  }
  // per-pair buffer of the transposed near field
  if (acc > 0 && op->f.built) CK(cudaMalloc(&op->f.nadj, sizeof(cx<float>) * acc * 12));
  if (acc > 0 && op->d.built) CK(cudaMalloc(&op->d.nadj, sizeof(cx<double>) * acc * 12));
  const int64_t work = acc * op->q;
  if (work > 0) {
    k_near_corr<double><<<(int)cdiv(work, 128), 128, 0, s>>>(
        op->tri, op->qp, op->qw, op->base, op->d.L, op->d.dL, op->noff, op->nsrc, nt, acc, op->q, op->p, op->ke,
        op->ki, op->gspatial[0], op->gspatial[1], op->P[0], op->P[1], op->P[2], op->d.near, op->f.near);
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(s));
  cudaFree(cnt);
  for (int med = 0; med < 2; ++med) {
    cudaFree(op->gspatial[med]);
    op->gspatial[med] = nullptr;
  }
  // reverse list for the transposed near field: the pairs of each source
  // triangle, ascending pair index
  if (acc > 0) {
    std::vector<int32_t> hs(acc), rc(nt + 1, 0), rp(acc);
    CK(cudaMemcpy(hs.data(), op->nsrc, sizeof(int32_t) * acc, cudaMemcpyDeviceToHost));
    for (int64_t j = 0; j < acc; ++j) ++rc[hs[j] + 1];
    for (int64_t t = 0; t < nt; ++t) rc[t + 1] += rc[t];
    std::vector<int32_t> cur(rc.begin(), rc.end() - 1);
    for (int64_t j = 0; j < acc; ++j) rp[cur[hs[j]]++] = (int32_t)j;
    CK(cudaMalloc(&op->roff, sizeof(int32_t) * (nt + 1)));
    CK(cudaMalloc(&op->rpair, sizeof(int32_t) * acc));
    CK(cudaMemcpy(op->roff, rc.data(), sizeof(int32_t) * (nt + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(op->rpair, rp.data(), sizeof(int32_t) * acc, cudaMemcpyHostToDevice));
  }
  return SCABEM_OK;
}

int setup_sigma_monomial(scabem_op* op, int nseg, const double* seg, cudaStream_t s) {
  double* dseg = nullptr;
  if (nseg > 0) {
    CK(cudaMalloc(&dseg, sizeof(double) * 6 * nseg));
    CK(cudaMemcpyAsync(dseg, seg, sizeof(double) * 6 * nseg, cudaMemcpyHostToDevice, s));
  }
  k_sigma_monomial<<<(int)cdiv(op->Q, 256), 256, 0, s>>>(op->qp, op->Q, nseg, dseg, op->d.sig, op->f.sig, op->sig64);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  if (dseg) cudaFree(dseg);
  return setup_precond(op, s);  // the absorber blocks depend on sigma
}

int setup_sigma_bspline(scabem_op* op, double x0, double L, int axis, int ncoef, const double* coef, cudaStream_t s) {
  double* dc = nullptr;
  CK(cudaMalloc(&dc, sizeof(double) * ncoef));
  CK(cudaMemcpyAsync(dc, coef, sizeof(double) * ncoef, cudaMemcpyHostToDevice, s));
  k_sigma_bspline<<<(int)cdiv(op->Q, 256), 256, 0, s>>>(op->qp, op->Q, x0, L, axis, ncoef, dc, op->d.sig, op->f.sig,
                                                        op->sig64);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  cudaFree(dc);
  return setup_precond(op, s);
}

int setup_sigma_values(scabem_op* op, const double* per_q_host, cudaStream_t s) {
  double* tmp = nullptr;
  CK(cudaMalloc(&tmp, sizeof(double) * op->Q));
  CK(cudaMemcpyAsync(tmp, per_q_host, sizeof(double) * op->Q, cudaMemcpyHostToDevice, s));
  k_sigma_copy<<<(int)cdiv(op->Q, 256), 256, 0, s>>>(tmp, op->Q, op->d.sig, op->f.sig, op->sig64);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  cudaFree(tmp);
  return setup_precond(op, s);
}
