// Device code of liblbs: the fused per-iteration update of the moment-chain
// lattice Boltzmann method for non-linear solids (arXiv 2502.00920,
// Algorithm 1), plus the initialisation, field-output, monitor and probe
// kernels.  Included by kernels_fp64.cu / kernels_fp32.cu / kernels_fp16.cu,
// each of which instantiates it for one storage precision.
//
// State between iterations (per node): the post-collision distributions g
// (9 values) and the displacement u.  One fused kernel per iteration k:
//   1. on the tile plus a 2-node halo: pull-stream g_k (bounce-back /
//      anti-bounce-back where the source lies outside, Eq. bbcon / abbcon)
//      and advance u with the trapezoidal rule,
//        u_{k+1} = u_k + dt/(2 rho0) (sum_q c_q g_k,q + sum_q c_q f_{k+1,q}),
//      which equals dt/(2 rho0) (j(t+dt) + j(t)) of Sect. 3.2 because the
//      collision adds dt S to the first moment;
//   2. on the tile plus a 1-node halo: H = grad u_{k+1} by finite
//      differences and N = P(H) + Pi(H) (Eq. source);
//   3. on the tile: S = rho0 b + div N, BGK collision of f_{k+1} with the
//      forcing term (Alg. 1), store g_{k+1} and u_{k+1}; on wall nodes store
//      N for the Neumann rule of the next iteration.
// The collision at t therefore uses S(u(t)), as Sect. 3.1 requires.
#pragma once
#include <cuda_fp16.h>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lbs_internal.h"

namespace lbs {

// ------------------------------------------------------------------ D2Q9
// Tab. 1: c_q = c (ex(q), ey(q)) (lbs_tiles.h); weights 4/9, 1/9 (axes), 1/36 (diagonals)
template <class R>
__host__ __device__ constexpr R wq(int q) { return q == 0 ? R(4) / R(9) : (q <= 4 ? R(1) / R(9) : R(1) / R(36)); }

// ------------------------------------------------------------------ precision
struct F64 {
  using real = double;
  using gs = double;
  using us = double2;
  static constexpr int id = LBS_FP64;
};
struct F32 {
  using real = float;
  using gs = float;
  using us = float4;  // (hi_x, hi_y, lo_x, lo_y): u = hi + lo
  static constexpr int id = LBS_FP32;
};
struct F16 {
  using real = float;
  using gs = __half;  // g * 2^gshift
  using us = float4;
  static constexpr int id = LBS_FP16S;
};

__device__ __forceinline__ double gload(const double *p, size_t i, double) { return __ldg(p + i); }
__device__ __forceinline__ float gload(const float *p, size_t i, float) { return __ldg(p + i); }
// FP16 storage: the kernels work in units of g * 2^gshift (exact power-of-two
// scaling), so loads and stores only convert
__device__ __forceinline__ float gload(const __half *p, size_t i, float) { return __half2float(__ldg(p + i)); }
__device__ __forceinline__ void gstore(double *p, size_t i, double v, double) { p[i] = v; }
__device__ __forceinline__ void gstore(float *p, size_t i, float v, float) { p[i] = v; }
__device__ __forceinline__ void gstore(__half *p, size_t i, float v, float) { p[i] = __float2half_rn(v); }

// FP16 storage holds g in units of g * 2^gshift (an exact power-of-two
// scaling); the wider types have gshift = 0 and get the factors as
// compile-time ones.  gscale<gs, R>(P) = 2^gshift, gscale_inv = 2^-gshift.
template <class G, class R>
__host__ __device__ __forceinline__ R gscale(const Params &P) {
  if constexpr (sizeof(G) == 2) return (R)ldexp(1.0, P.gshift);
  else return R(1);
}
template <class G, class R>
__host__ __device__ __forceinline__ R gscale_inv(const Params &P) {
  if constexpr (sizeof(G) == 2) return (R)ldexp(1.0, -P.gshift);
  else return R(1);
}

// difference of two displacement records, as the compute type
__device__ __forceinline__ void udiff(const double2 &a, const double2 &b, double &dx, double &dy) {
  dx = a.x - b.x;
  dy = a.y - b.y;
}
// hi parts of neighbouring nodes are close, so their difference is exact or
// correctly rounded; the lo parts carry what lies below the hi ulp
__device__ __forceinline__ void udiff(const float4 &a, const float4 &b, float &dx, float &dy) {
  dx = (a.x - b.x) + (a.z - b.z);
  dy = (a.y - b.y) + (a.w - b.w);
}

__device__ __forceinline__ double2 uadd(const double2 &u, double dx, double dy) { return make_double2(u.x + dx, u.y + dy); }

// compensated accumulation: (hi, lo) + d.  hi takes the rounded sum; the
// rounding error of hi + d (two-sum, Knuth: exact) is added to lo, which so
// gathers the errors of all increments; the value is hi + lo.  (lo is not
// renormalised into hi: it stays a small multiple of hi's rounding unit, far
// inside its own range, and the finite differences take both parts.)
__device__ __forceinline__ void pair_add(float &hi, float &lo, float d) {
  const float s = hi + d;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (d - bp);
  lo = lo + e;
  hi = s;
}
__device__ __forceinline__ float4 uadd(const float4 &u, float dx, float dy) {
  float4 r = u;
  pair_add(r.x, r.z, dx);
  pair_add(r.y, r.w, dy);
  return r;
}

// u + kap * (mx, my): one rounding per component in double; the float pair
// adds the rounded increment compensated
__device__ __forceinline__ double2 uadd_k(const double2 &u, double kap, double mx, double my) {
  return make_double2(fma(kap, mx, u.x), fma(kap, my, u.y));
}
__device__ __forceinline__ float4 uadd_k(const float4 &u, float kap, float mx, float my) {
  return uadd(u, kap * mx, kap * my);
}

__device__ __forceinline__ double2 u_value(const double2 &u) { return u; }
__device__ __forceinline__ double2 u_value(const float4 &u) {
  return make_double2((double)u.x + (double)u.z, (double)u.y + (double)u.w);
}
__device__ __forceinline__ void u_make(double x, double y, double2 &out) { out = make_double2(x, y); }
__device__ __forceinline__ void u_make(double x, double y, float4 &out) {
  float hx = (float)x, hy = (float)y;
  out = make_float4(hx, hy, (float)(x - (double)hx), (float)(y - (double)hy));
}

// a * b + c with a single rounding.  The library is compiled without
// implicit contraction (nvcc --fmad=false): every product and sum not written
// with fmr rounds on its own, so the rounding of each expression is fixed by
// the source, and every tile shape, frame and batch kernel computes a node
// with the same operations whatever the compiler inlines or schedules.
__host__ __device__ __forceinline__ float fmr(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ double fmr(double a, double b, double c) { return fma(a, b, c); }

// First moment sum_q e_q v_q of nine populations (index 0 unused), from the
// differences of opposite pairs.  In a near-static state each population is
// close to its opposite, so every pair difference is exact (Sterbenz) and the
// sum rounds relative to the momentum, not to the populations it is a small
// difference of: in single precision the displacement increment then keeps
// its relative accuracy over long, slow loadings.
template <class R>
__host__ __device__ __forceinline__ void first_moment(const R v[9], R &mx, R &my) {
  const R d57 = v[5] - v[7], d68 = v[6] - v[8];
  mx = (v[1] - v[3]) + (d57 - d68);
  my = (v[2] - v[4]) + (d57 + d68);
}

// ------------------------------------------------------------------ material
// N(H) = P(H) + Pi(H), Pi(H) = -mu (H + H^T + tr H I), written so that no
// term cancels at small strain (Sect. 4 laws, rearranged):
//   SVK: N = (lam trE - mu trH) I + mu H^T H + H S,  S = lam trE I + mu (H + H^T + H^T H)
//   NH : with a = J - 1 = trH + detH, K = trH I - H^T (cof F = I + K),
//        N = (mu/J) (-a H^T + (a - (2 + a) trH) I) + lam a (a + 2) / (2 J) (I + K)
//   LE : N = (lam - mu) trH I
// H = (H11, H12, H21, H22), H_ab = d u_a / d X_b.  Returns false, with N
// unset, for neo-Hooke where J < jmin (the caller then evaluates the law in
// a wider type); the default jmin never refuses.
template <class R>
__host__ __device__ inline bool constitutive_n(int model, R lam, R mu, const R H[4], R N[4], R jmin = R(-INFINITY)) {
  const R h11 = H[0], h12 = H[1], h21 = H[2], h22 = H[3];
  const R trH = h11 + h22;
  if (model == LBS_LE) {
    const R d = (lam - mu) * trH;
    N[0] = d;
    N[1] = R(0);
    N[2] = R(0);
    N[3] = d;
  } else if (model == LBS_SVK) {
    // H^T H
    const R c11 = fmr(h11, h11, h21 * h21), c12 = fmr(h11, h12, h21 * h22), c22 = fmr(h12, h12, h22 * h22);
    const R trE = fmr(R(0.5), c11 + c22, trH);
    const R s11 = fmr(lam, trE, mu * (R(2) * h11 + c11));
    const R s12 = mu * ((h12 + h21) + c12);
    const R s22 = fmr(lam, trE, mu * (R(2) * h22 + c22));
    const R d = fmr(lam, trE, -(mu * trH));
    const R mc12 = mu * c12;
    N[0] = fmr(h12, s12, fmr(h11, s11, fmr(mu, c11, d)));
    N[1] = fmr(h12, s22, fmr(h11, s12, mc12));
    N[2] = fmr(h22, s12, fmr(h21, s11, mc12));
    N[3] = fmr(h22, s22, fmr(h21, s12, fmr(mu, c22, d)));
  } else {  // LBS_NH
    const R detH = fmr(h11, h22, -(h12 * h21));
    const R a = trH + detH;
    const R J = R(1) + a;
    if (J < jmin) return false;
    const R iJ = R(1) / J;
    const R m = mu * iJ;
    const R l = R(0.5) * lam * a * (a + R(2)) * iJ;
    const R diag = m * fmr(-(R(2) + a), trH, a);
    const R ma = m * a;
    // I + K = [[1 + h22, -h21], [-h12, 1 + h11]]
    N[0] = fmr(-ma, h11, fmr(l, R(1) + h22, diag));
    N[1] = -((ma + l) * h21);
    N[2] = -((ma + l) * h12);
    N[3] = fmr(-ma, h22, fmr(l, R(1) + h11, diag));
  }
  return true;
}

// N in the compute type; the FP32 kernels evaluate neo-Hooke in double where
// J < 1/2 (near det F -> 0 the 1/J terms lose float accuracy)
template <class R>
__device__ __forceinline__ void material(const Params &P, R lam, R mu, const R H[4], R N[4]) {
  if constexpr (sizeof(R) == 4) {
    if (!constitutive_n<R>(P.model, lam, mu, H, N, R(0.5))) {
      double Hd[4] = {H[0], H[1], H[2], H[3]}, Nd[4];
      constitutive_n<double>(P.model, P.lam, P.mu, Hd, Nd);
      for (int m = 0; m < 4; ++m) N[m] = (R)Nd[m];
    }
  } else {
    constitutive_n<R>(P.model, lam, mu, H, N);
  }
}

// ------------------------------------------------------------------ loads
// prescribed boundary value amp * s(k) of edge e at iteration k
__device__ inline void edge_value(const Params &P, int e, int64_t k, double out[2]) {
  const double t = P.eunit[e] == LBS_TIME ? (double)k * P.dt : (double)k;
  const double t0 = P.et0[e], t1 = P.et1[e], span = t1 - t0;
  double f;
  switch (P.eshape[e]) {
    case LBS_CONST: f = 1.0; break;
    case LBS_LINEAR_RAMP: f = fmin(fmax((t - t0) / span, 0.0), 1.0); break;
    case LBS_SIN2_RAMP: {
      const double sn = sin(0.5 * M_PI * fmin(fmax((t - t0) / span, 0.0), 1.0));
      f = sn * sn;
      break;
    }
    case LBS_HALF_SINE: f = (t >= t0 && t < t1) ? sin(M_PI * (t - t0) / span) : 0.0; break;
    case LBS_RICKER: {
      const double d = t - t0;
      f = t < t1 ? (1.0 - d * d / P.es[e]) * exp(-0.5 * d * d / P.es[e]) : 0.0;
      break;
    }
    case LBS_DISP_RAMP:
      f = (t >= t0 && t < t1) ? P.rho0 / (P.eunit[e] == LBS_TIME ? span : span * P.dt) : 0.0;
      break;
    default: f = 0.0;
  }
  out[0] = P.eamp[e][0] * f;
  out[1] = P.eamp[e][1] * f;
}

// ------------------------------------------------------------------ boundary rules
// Pull-form boundary rules at a wall node (x, y): for every direction q whose
// source x - c_q dt lies outside the lattice (bit q of `mask`), the outgoing
// link qbar = opp(q) crosses a wall and f_q(x) is set from the node's own
// post-collision g (Sect. 3.3):
//   Dirichlet (Eq. bbcon):   f_q = g_qbar + 2 w_q c_q . j* / cs^2
//   Neumann   (Eq. abbcon):  f_q = -g_qbar + 2 w_q (r + (Pi* - r cs^2 I):(c_q c_q - cs^2 I) / (2 cs^4))
// with r and the tangential Pi entry from the node's own moments, and the
// normal row/column of Pi* from -T* + (P + Pi(H)) N (N of this node, stored by
// the previous iteration).  Each link uses the wall it crosses; a diagonal link
// crossing two walls is Dirichlet if either wall is (mean j* if both), else
// its Pi* takes Pi*_xx from the x wall, Pi*_yy from the y wall and the mean of
// the two shear entries.
// Under two-point extrapolation (P.extrap) each of these node values v is
// carried to the wall(s) the link crosses as v + (v - v_in)/2 per crossed
// wall, v_in the value at the next node inwards along that wall's normal: r
// and Pi from that node's own g, N from the side array's second layer.
template <class R, class G, bool LIN>
__device__ void wall_rules(const Params &P, const R *bnd, const G *g, const double (*sev)[2], int x, int y,
                           const R g0[9], unsigned mask, R f[9], R gsc) {
  int xw, yw;
  walls_of(P, x, y, xw, yw);
  const bool xn = xw >= 0 && P.etype[xw] == LBS_NEUMANN;
  const bool yn = yw >= 0 && P.etype[yw] == LBS_NEUMANN;
  // Pi*/cs^2 from N and T* is brought into the units of g (times gsc)
  const R ics2 = (R)P.inv_cs2 * gsc;
  // own moments (collision leaves r and Pi unchanged): r, A = Pi / cs^2 = 3 sum e e g
  R r = 0, mxx = 0, mxy = 0, myy = 0;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    r += g0[q];
    mxx += R(ex(q) * ex(q)) * g0[q];
    mxy += R(ex(q) * ey(q)) * g0[q];
    myy += R(ey(q) * ey(q)) * g0[q];
  }
  // Pi*/cs^2 pieces: the node's own moment (entries extrapolated to the wall)
  // and the normal column of each Neumann wall the node sits on
  const R Axx_o = R(3) * mxx, Axy_o = R(3) * mxy, Ayy_o = R(3) * myy;
  R Axx_x = 0, axy_x = 0, Ayy_y = 0, axy_y = 0;
  if (xn) {
    const R *Nn = bnd + side_entry(P, 0, xw, y);  // N11, N12, N21, N22
    const double *T = sev[xw];
    const R s = (xw == kRight) ? R(1) : R(-1);
    Axx_x = (Nn[0] - s * (R)T[0]) * ics2;
    axy_x = (Nn[2] - s * (R)T[1]) * ics2;
  }
  if (yn) {
    const R *Nn = bnd + side_entry(P, 0, yw, x);
    const double *T = sev[yw];
    const R s = (yw == kTop) ? R(1) : R(-1);
    Ayy_y = (Nn[3] - s * (R)T[1]) * ics2;
    axy_y = (Nn[1] - s * (R)T[0]) * ics2;
  }
  // two-point extrapolation: half the differences own - inner of r, A and N
  // for the x wall (dX, nX) and the y wall (dY, nY) the node sits on (a
  // lattice without the setting has no second side-array layer to read).
  R dX[4] = {0, 0, 0, 0}, dY[4] = {0, 0, 0, 0}, nX[4] = {0, 0, 0, 0}, nY[4] = {0, 0, 0, 0};
  if (LIN && P.extrap) {
    const size_t plane = (size_t)P.ny * P.pitch;
    const R own[4] = {r, Axx_o, Axy_o, Ayy_o};
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int e = w == 0 ? xw : yw;
      if (e < 0) continue;
      int xi, yi;
      inner_node(e, x, y, xi, yi);
      const size_t idx = (size_t)yi * P.pitch + xi;
      R ri = 0, ixx = 0, ixy = 0, iyy = 0;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const R v = gload(g, q * plane + idx, R(1));
        ri += v;
        ixx += R(ex(q) * ex(q)) * v;
        ixy += R(ex(q) * ey(q)) * v;
        iyy += R(ey(q) * ey(q)) * v;
      }
      const R in[4] = {ri, R(3) * ixx, R(3) * ixy, R(3) * iyy};
      const int pos = w == 0 ? y : x;
      const R *N0 = bnd + side_entry(P, 0, e, pos);
      const R *N1 = bnd + side_entry(P, 1, e, pos);
      R *d = w == 0 ? dX : dY;
      R *n = w == 0 ? nX : nY;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        d[m] = R(0.5) * (own[m] - in[m]);
        n[m] = R(0.5) * (N0[m] - N1[m]) * ics2;
      }
    }
  }
  const R cj = (R)(P.c * P.inv_cs2) * gsc;
#pragma unroll
  for (int q = 1; q < 9; ++q) {
    if (!(mask & (1u << q))) continue;
    bool ox, oy;
    link_crosses(P, x, y, q, ox, oy);
    const bool dxw = ox && P.etype[xw] == LBS_DIRICHLET;
    const bool dyw = oy && P.etype[yw] == LBS_DIRICHLET;
    const int qb = opp(q);
    if (dxw || dyw) {
      double js[2];
      if (dxw && dyw) {
        const double *a = sev[xw], *b = sev[yw];
        js[0] = 0.5 * (a[0] + b[0]);
        js[1] = 0.5 * (a[1] + b[1]);
      } else {
        js[0] = sev[dxw ? xw : yw][0];
        js[1] = sev[dxw ? xw : yw][1];
      }
      f[q] = g0[qb] + R(2) * wq<R>(q) * cj * (R(ex(q)) * (R)js[0] + R(ey(q)) * (R)js[1]);
    } else if constexpr (!LIN) {
      // Pi* of the wall(s) this link crosses
      const R Axx = ox ? Axx_x : Axx_o;
      const R Ayy = oy ? Ayy_y : Ayy_o;
      const R Axy = (ox && oy) ? R(0.5) * (axy_x + axy_y) : (ox ? axy_x : axy_y);
      const R e2 = R(ex(q) * ex(q) + ey(q) * ey(q));
      const R eAe = R(ex(q) * ex(q)) * Axx + R(2 * ex(q) * ey(q)) * Axy + R(ey(q) * ey(q)) * Ayy;
      f[q] = -g0[qb] + wq<R>(q) * (R(4) * r - R(3) * r * e2 + R(3) * eAe - (Axx + Ayy));
    } else {
      // the same with the values extrapolated across the crossed walls only
      const R ax = ox ? R(1) : R(0), ay = oy ? R(1) : R(0);
      auto e = [&](int m, const R *a, const R *b) { return ax * a[m] + ay * b[m]; };
      const R rw = r + e(0, dX, dY);
      const R Axx_e = Axx_o + e(1, dX, dY), Axy_e = Axy_o + e(2, dX, dY), Ayy_e = Ayy_o + e(3, dX, dY);
      const R axx_x = Axx_x + e(0, nX, nY), axy_xe = axy_x + e(2, nX, nY);
      const R ayy_y = Ayy_y + e(3, nX, nY), axy_ye = axy_y + e(1, nX, nY);
      const R Axx = ox ? axx_x : Axx_e;
      const R Ayy = oy ? ayy_y : Ayy_e;
      const R Axy = (ox && oy) ? R(0.5) * (axy_xe + axy_ye) : (ox ? axy_xe : (oy ? axy_ye : Axy_e));
      const R e2 = R(ex(q) * ex(q) + ey(q) * ey(q));
      const R eAe = R(ex(q) * ex(q)) * Axx + R(2 * ex(q) * ey(q)) * Axy + R(ey(q) * ey(q)) * Ayy;
      f[q] = -g0[qb] + wq<R>(q) * (R(4) * rw - R(3) * rw * e2 + R(3) * eAe - (Axx + Ayy));
    }
  }
}

// ------------------------------------------------------------------ collision
// BGK collision with forcing (Alg. 1): g = f - (f - feq)/tau + (1 - 1/(2 tau)) psi dt.
// feq (Eq. feq, second-order Hermite) takes r, j = c sum e f + dt/2 S and
// Pi = sum c c f from f itself, so f - feq has no component along r, j or Pi:
// written out in the populations it is, with the pair sums and differences
//   s13 = f1 + f3, d13 = f1 - f3 (likewise 24, 57, 68),
// one even combination Q = f0 - 2 (s13 + s24) + 4 (s57 + s68), giving
//   (f - feq)_q even part = w_q Q chi_q,  chi = 1/4 (rest), -1/2 (axes), 1 (diagonals),
// and four odd ones (the odd parts of f - feq on the axis and diagonal pairs)
//   ox = d13/6 - (d57 - d68)/3,   oy = d24/6 - (d57 + d68)/3,
//   o57 = d57/3 - (d13 + d24)/12, o68 = d68/3 - (d24 - d13)/12,
// each less the dt/2 S part of j, which combines with the forcing term
// (1 - 1/(2 tau)) psi dt into w_q sigma e_q.S per population (sigma = c dt / cs^2;
// its first moment is sigma S / 3 = dt S / c, the momentum the source adds).
// So g_q = f_q - omega (f - feq)_q + w_q sigma e_q.S.  The same algebra as
// the literal moment form, but every intermediate is of the size of the
// populations, so single-precision rounding stays at the level of the stored
// values instead of that of the second moments.
// Per-thread constants of the collision: -omega, the relaxation of the even
// part per unit Q for the axis (omega/18) and diagonal (-omega/36)
// populations, and the forcing weights sigma/9 and sigma/36 times the storage
// scale of g (the source arrives unscaled).
template <class R>
struct CollideK {
  R mo, m6, m9, m12, a1, a5, s9, s36;
};
template <class R>
__device__ __forceinline__ CollideK<R> collide_k(R omega, R sigma, R scl) {
  const R ss = sigma * scl;
  return {-omega,
          -omega * (R(1) / R(6)),
          -omega * (R(1) / R(9)),
          -omega * (R(1) / R(12)),
          omega * (R(1) / R(18)),
          -omega * (R(1) / R(36)),
          ss * (R(1) / R(9)),
          ss * (R(1) / R(36))};
}

// Each opposite pair takes the even relaxation A = Q a1 or Q a5 (the same for
// both) and the odd part b = -omega o + forcing with opposite signs:
// g = (f + A) +- b; in FP64 the product Q a is fused into the population's
// own add, g = fma(Q, a, f) +- b.
template <class R>
__device__ __forceinline__ void collide(R f[9], R Sx, R Sy, const CollideK<R> &K) {
  const R s13 = f[1] + f[3], s24 = f[2] + f[4], s57 = f[5] + f[7], s68 = f[6] + f[8];
  const R d13 = f[1] - f[3], d24 = f[2] - f[4], d57 = f[5] - f[7], d68 = f[6] - f[8];
  // (the products by 2 and 4 are exact)
  const R Q = fmr(R(4), s57 + s68, fmr(R(-2), s13 + s24, f[0]));
  const R fx = Sx * K.s9, fy = Sy * K.s9;
  const R f57 = (Sx + Sy) * K.s36, f68 = (Sy - Sx) * K.s36;
  const R A1 = Q * K.a1, A5 = Q * K.a5;  // (single precision; unused in FP64)
  R bx, by, b57, b68;
  if constexpr (sizeof(R) == 8) {
    // the odd parts, ox = (d13 - 2 (d57 - d68)) / 6 and so on, enter only as
    // -omega times them: the division goes into that factor (the products by
    // 2 and 4 are exact), four FP64 operations fewer per node
    const R tx = fmr(R(-2), d57 - d68, d13), ty = fmr(R(-2), d57 + d68, d24);
    const R t57 = fmr(R(4), d57, -(d13 + d24)), t68 = fmr(R(4), d68, -(d24 - d13));
    bx = fmr(tx, K.m6, fx);
    by = fmr(ty, K.m6, fy);
    b57 = fmr(t57, K.m12, f57);
    b68 = fmr(t68, K.m12, f68);
  } else {
    // (single precision keeps the odd parts themselves: the form above
    // measured slower for FP16 storage, whose kernel is issue-bound)
    const R c3 = R(1) / R(3), c6 = R(1) / R(6), c12 = R(1) / R(12);
    const R ox = fmr(d13, c6, -((d57 - d68) * c3));
    const R oy = fmr(d24, c6, -((d57 + d68) * c3));
    const R o57 = fmr(d57, c3, -((d13 + d24) * c12));
    const R o68 = fmr(d68, c3, -((d24 - d13) * c12));
    bx = fmr(K.mo, ox, fx);
    by = fmr(K.mo, oy, fy);
    b57 = fmr(K.mo, o57, f57);
    b68 = fmr(K.mo, o68, f68);
  }
  if constexpr (sizeof(R) == 8) {
    // three FP64 multiplies fewer per node
    f[0] = fmr(Q, K.m9, f[0]);
    f[1] = fmr(Q, K.a1, f[1]) + bx;
    f[3] = fmr(Q, K.a1, f[3]) - bx;
    f[2] = fmr(Q, K.a1, f[2]) + by;
    f[4] = fmr(Q, K.a1, f[4]) - by;
    f[5] = fmr(Q, K.a5, f[5]) + b57;
    f[7] = fmr(Q, K.a5, f[7]) - b57;
    f[6] = fmr(Q, K.a5, f[6]) + b68;
    f[8] = fmr(Q, K.a5, f[8]) - b68;
  } else {
    // (single precision keeps the separate products: the fused form takes
    // the FP16-storage TMA kernel past 64 registers)
    f[0] = fmr(K.mo, Q * (R(1) / R(9)), f[0]);
    f[1] = (f[1] + A1) + bx;
    f[3] = (f[3] + A1) - bx;
    f[2] = (f[2] + A1) + by;
    f[4] = (f[4] + A1) - by;
    f[5] = (f[5] + A5) + b57;
    f[7] = (f[7] + A5) - b57;
    f[6] = (f[6] + A5) + b68;
    f[8] = (f[8] + A5) - b68;
  }
}

// ------------------------------------------------------------------ tiles
// A thread block owns a TX x TY tile of nodes; NTY thread rows, each thread
// handles CPT = TY / NTY nodes of one column.  Shared memory holds u_{k+1}
// on the tile plus a 2-node halo (R2) and N on the tile plus a 1-node halo (R1).
// (geometry and index arithmetic in lbs_tiles.h: TileGeom, ring_pos, locate)
template <class Pr, int TX_, int TY_, int NTY_>
struct TileCfg : TileGeom<TX_, TY_, NTY_> {
  using G = TileGeom<TX_, TY_, NTY_>;
  using real = typename Pr::real;
  using us = typename Pr::us;
  using gs = typename Pr::gs;
  struct Smem {
    us u[G::R2H][G::R2W];
    real n[4][G::R1H][G::R1W];
  };
};

// Stream into node (x, y) (already wrapped into the lattice) and return the
// first moments sum_q e_q g_q (own node, post-collision at k) and
// sum_q e_q f_q (streamed, at k + 1).  EDGE: wrap, walls and boundary rules;
// LIN: the two-point wall extrapolation (lattices with P.extrap set).
template <class Pr, bool EDGE, bool LIN>
__device__ __forceinline__ void gather(const Params &P, const typename Pr::gs *__restrict__ g, const typename Pr::real *bnd,
                                       const double (*sev)[2], int x, int y, typename Pr::real inv,
                                       typename Pr::real f[9], typename Pr::real &gx, typename Pr::real &gy,
                                       typename Pr::real gsc) {
  using R = typename Pr::real;
  const size_t plane = (size_t)P.ny * P.pitch;
  const size_t idx = (size_t)y * P.pitch + x;
  R g0[9];
  // every streaming source inside the lattice without wrapping: loads at
  // fixed offsets, no boundary rule (all interior tiles, and most nodes of
  // the frame tiles, which lie within three nodes of a wall or of the end)
  if (!EDGE || (x >= 1 && x <= P.nx - 2 && y >= 1 && y <= P.ny - 2)) {
#pragma unroll
    for (int q = 0; q < 9; ++q) f[q] = gload(g, q * plane + idx - ex(q) - (ptrdiff_t)ey(q) * P.pitch, inv);
#pragma unroll
    for (int q = 1; q < 9; ++q) g0[q] = gload(g, q * plane + idx, inv);
    g0[0] = 0;
  } else if constexpr (sizeof(R) == 8) {
    // FP64: loads between the branches (the batched form below takes the
    // frame kernel past 128 registers, halving its blocks per SM)
    unsigned mask = 0;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      g0[q] = gload(g, q * plane + idx, inv);
      int sx, sy;
      if (!stream_source(P, x, y, q, sx, sy)) {
        mask |= 1u << q;
        f[q] = 0;
      } else {
        f[q] = gload(g, q * plane + (size_t)sy * P.pitch + sx, inv);
      }
    }
    if (mask) wall_rules<R, typename Pr::gs, LIN>(P, bnd, g, sev, x, y, g0, mask, f, gsc);
  } else {
    // source of each population first (the node itself where the source
    // lies outside the lattice), then all eighteen loads without branches in
    // between, so that they are in flight together
    unsigned mask = 0;
    size_t src[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      int sx, sy;
      const bool in = stream_source(P, x, y, q, sx, sy);
      if (!in) mask |= 1u << q;
      src[q] = in ? (size_t)sy * P.pitch + sx : idx;
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      g0[q] = gload(g, q * plane + idx, inv);
      f[q] = gload(g, q * plane + src[q], inv);
    }
#pragma unroll
    for (int q = 0; q < 9; ++q)
      if (mask & (1u << q)) f[q] = 0;
    if (mask) wall_rules<R, typename Pr::gs, LIN>(P, bnd, g, sev, x, y, g0, mask, f, gsc);
  }
  first_moment(g0, gx, gy);
}

// store N of wall node (x, y) into the side array entries of its walls
template <class R>
__device__ __forceinline__ void store_wall_n(const Params &P, R *bnd, int x, int y, const R N[4]) {
  int xw, yw;
  walls_of(P, x, y, xw, yw);
  if (xw >= 0) {
    R *d = bnd + side_entry(P, 0, xw, y);
    for (int m = 0; m < 4; ++m) d[m] = N[m];
  }
  if (yw >= 0) {
    R *d = bnd + side_entry(P, 0, yw, x);
    for (int m = 0; m < 4; ++m) d[m] = N[m];
  }
}

// under two-point extrapolation: store N of node (x, y) into the side array's
// second layer for each wall it lies one step inwards from
template <class R>
__device__ __forceinline__ void store_inner_n(const Params &P, R *bnd, int x, int y, const R N[4]) {
  int e[4], pos[4];
  const int n = inner_entries(P, x, y, e, pos);
  for (int i = 0; i < n; ++i) {
    R *d = bnd + side_entry(P, 1, e[i], pos[i]);
    for (int m = 0; m < 4; ++m) d[m] = N[m];
  }
}

// d/dX of a shared-memory row: central inside, one-sided on the first and
// last node of a walled axis (Sect. 3.2); `lo`/`hi` say the node is such a
// wall node.  Returns the difference already divided by the spacing.
template <class C, bool EDGE>
struct Fd {
  using R = typename C::real;
  // H at R1 position (rx, ry) from su (R2 coords = R1 + 1)
  static __device__ __forceinline__ void grad(const typename C::Smem &sm, const Params &P, int rx, int ry, int gxn,
                                              int gyn, R idx_, R H[4]) {
    R dxx, dxy, dyx, dyy;  // d u_x/dx, d u_y/dx, d u_x/dy, d u_y/dy
    const int cx = rx + 1, cy = ry + 1;
    int xa, xb, ya, yb;
    bool onex, oney;
    fd_taps<EDGE>(P, cx, cy, gxn, gyn, xa, xb, ya, yb, onex, oney);
    const R sx = onex ? idx_ : R(0.5) * idx_, sy = oney ? idx_ : R(0.5) * idx_;
    udiff(sm.u[cy][xa], sm.u[cy][xb], dxx, dxy);
    udiff(sm.u[ya][cx], sm.u[yb][cx], dyx, dyy);
    H[0] = dxx * sx;
    H[1] = dyx * sy;
    H[2] = dxy * sx;
    H[3] = dyy * sy;
  }
  // S = div N + (sbx, sby) at R1 position (rx, ry) of a tile node
  static __device__ __forceinline__ void div(const typename C::Smem &sm, const Params &P, int rx, int ry, int gxn,
                                             int gyn, R idx_, R sbx, R sby, R &Sx, R &Sy) {
    int xa, xb, ya, yb;
    bool onex, oney;
    fd_taps<EDGE>(P, rx, ry, gxn, gyn, xa, xb, ya, yb, onex, oney);
    const R sx = onex ? idx_ : R(0.5) * idx_, sy = oney ? idx_ : R(0.5) * idx_;
    Sx = fmr(sm.n[0][ry][xa] - sm.n[0][ry][xb], sx, fmr(sm.n[1][ya][rx] - sm.n[1][yb][rx], sy, sbx));
    Sy = fmr(sm.n[2][ry][xa] - sm.n[2][ry][xb], sx, fmr(sm.n[3][ya][rx] - sm.n[3][yb][rx], sy, sby));
  }
};

// phase 2: N over R1 from u in shared memory; N of own-tile wall nodes goes
// to the side array (and, with LIN on a lattice with P.extrap set, N of the
// nodes one step inwards to its second layer)
template <class C, bool EDGE, bool LIN = false>
__device__ __forceinline__ void phase_n(typename C::Smem &sm, const Params &P, int x0, int y0, typename C::real *bnd_out) {
  using R = typename C::real;
  const R lam = (R)P.lam, mu = (R)P.mu, idx_ = (R)P.inv_dx;
  for (int e = threadIdx.x; e < C::R1W * C::R1H; e += C::NT) {
    const int rx = e % C::R1W, ry = e / C::R1W;
    int gx = x0 - 1 + rx, gy = y0 - 1 + ry;
    if (EDGE && !locate(P, gx, gy)) continue;
    R H[4], N[4];
    Fd<C, EDGE>::grad(sm, P, rx, ry, gx, gy, idx_, H);
    material<R>(P, lam, mu, H, N);
#pragma unroll
    for (int m = 0; m < 4; ++m) sm.n[m][ry][rx] = N[m];
    if (EDGE && bnd_out && r1_own_node<C>(P, x0, y0, rx, ry)) {
      if (on_wall(P, gx, gy)) store_wall_n<R>(P, bnd_out, gx, gy, N);
      if (LIN && P.extrap) store_inner_n<R>(P, bnd_out, gx, gy, N);
    }
  }
}

// The fused iteration on one tile.
template <class C, bool EDGE, bool LIN = false>
__device__ __forceinline__ void step_tile(const Params &P, const StepPtrs &S, int x0, int y0) {
  using Pr_real = typename C::real;
  using R = Pr_real;
  using us = typename C::us;
  using gs = typename C::gs;
  __shared__ typename C::Smem sm;
  const gs *__restrict__ g = (const gs *)S.g_in;
  gs *__restrict__ go = (gs *)S.g_out;
  const us *__restrict__ u = (const us *)S.u_in;
  us *__restrict__ uo = (us *)S.u_out;
  const R *bnd = (const R *)S.b_in;
  const int64_t k = EDGE ? (*S.kptr + S.koff) : 0;
  // boundary values of the four edges at iteration k, evaluated once per
  // tile (the wall rules of every wall node read them)
  __shared__ double sev[4][2];
  if (EDGE) {
    if (S.sev) {
      if (threadIdx.x < 8) sev[threadIdx.x >> 1][threadIdx.x & 1] = S.sev[threadIdx.x];
    } else if (threadIdx.x < 4) {
      edge_value(P, threadIdx.x, k, sev[threadIdx.x]);
    }
    __syncthreads();
  }
  // g is held in units of g * 2^gshift (1 unless FP16 storage)
  const R inv = gscale_inv<typename C::gs, R>(P), scl = gscale<typename C::gs, R>(P);
  const R kap = (R)P.kappa * inv;
  const int tx = threadIdx.x % C::TX, ty = threadIdx.x / C::TX;

  // phase 1a: own nodes (keep the streamed populations).  In a tile that
  // overhangs the end of a periodic axis, the positions past the end are
  // wrapped neighbours that the stencils of the last nodes read: their u is
  // computed here too, but they are not stored.
  R f[C::CPT][9];
#pragma unroll
  for (int i = 0; i < C::CPT; ++i) {
    const int lx = tx, ly = ty + i * C::NTY;
    int x = x0 + lx, y = y0 + ly;
    if (EDGE && !locate(P, x, y)) continue;
    R gxm, gym;
    gather<typename C::PrT, EDGE, LIN>(P, g, bnd, sev, x, y, inv, f[i], gxm, gym, scl);
    R fx, fy;
    first_moment(f[i], fx, fy);
    sm.u[ly + 2][lx + 2] = uadd_k(u[(size_t)y * P.pitch + x], kap, gxm + fx, gym + fy);
  }
  // phase 1b: the 2-node frame (u only)
  for (int e = threadIdx.x; e < C::NRING; e += C::NT) {
    int rx, ry;
    ring_pos<C>(e, rx, ry);
    int x = x0 - 2 + rx, y = y0 - 2 + ry;
    if (EDGE && !locate(P, x, y)) continue;
    R ff[9], gxm, gym;
    gather<typename C::PrT, EDGE, LIN>(P, g, bnd, sev, x, y, inv, ff, gxm, gym, scl);
    R fx, fy;
    first_moment(ff, fx, fy);
    sm.u[ry][rx] = uadd_k(u[(size_t)y * P.pitch + x], kap, gxm + fx, gym + fy);
  }
  __syncthreads();
  phase_n<C, EDGE, LIN>(sm, P, x0, y0, (R *)S.b_out);
  __syncthreads();
  // phase 3: source, collision, store
  const size_t plane = (size_t)P.ny * P.pitch;
  const R idx_ = (R)P.inv_dx;
  const CollideK<R> K = collide_k<R>((R)P.omega, (R)P.sigma, scl);
  const R sbx = (R)(P.rho0 * P.body[0]), sby = (R)(P.rho0 * P.body[1]);
#pragma unroll
  for (int i = 0; i < C::CPT; ++i) {
    const int lx = tx, ly = ty + i * C::NTY;
    const int x = x0 + lx, y = y0 + ly;
    if (EDGE && (x >= P.nx || y >= P.ny)) continue;
    R Sx, Sy;
    Fd<C, EDGE>::div(sm, P, lx + 1, ly + 1, x, y, idx_, sbx, sby, Sx, Sy);
    collide<R>(f[i], Sx, Sy, K);
    const size_t idx = (size_t)y * P.pitch + x;
#pragma unroll
    for (int q = 0; q < 9; ++q) gstore(go, q * plane + idx, f[i][q], scl);
    uo[idx] = sm.u[ly + 2][lx + 2];
  }
}

template <class Pr, int TX, int TY, int NTY>
struct Cfg : TileCfg<Pr, TX, TY, NTY> {
  using PrT = Pr;
};

// interior tiles: R2 and its streaming sources lie inside, no wall, no wrap
template <class C>
__global__ void __launch_bounds__(C::NT) step_interior_kernel(const Params P, const StepPtrs S, int a_lo, int b_lo) {
  step_tile<C, false>(P, S, (a_lo + blockIdx.x) * C::TX, (b_lo + blockIdx.y) * C::TY);
}

// tiles of the frame around the interior block (walls, wrap, partial tiles):
// edge_tile in lbs_tiles.h

// With SPLIT, a frame tile of CPT nodes per thread is processed as CPT
// tiles of one node per thread by CPT blocks.  On a small lattice the frame
// tiles are few and the iteration waits on their latency; once there are
// more of them than SMs the pieces' extra halo work costs more than it saves
// (launch_edge chooses).
template <class C, bool SPLIT>
struct FrameCfg {
  using type = C;
};
template <class C>
struct FrameCfg<C, true> {
  using type = Cfg<typename C::PrT, C::TX, C::NTY, C::NTY>;
};

template <class C, bool LIN, bool SPLIT = false>
__global__ void __launch_bounds__(FrameCfg<C, SPLIT>::type::NT) step_edge_kernel(const Params P, const StepPtrs S,
                                                                                 int ntx, int a_lo, int a_hi,
                                                                                 int b_lo, int b_hi) {
  using H = typename FrameCfg<C, SPLIT>::type;
  constexpr int parts = C::TY / H::TY;
  int a, b;
  edge_tile(blockIdx.x / parts, ntx, a_lo, a_hi, b_lo, b_hi, a, b);
  step_tile<H, true, LIN>(P, S, a * C::TX, b * C::TY + (blockIdx.x % parts) * H::TY);
}

// the frame tiles of one iteration; the two-point wall extrapolation has its
// own instantiation so that the default frame kernel keeps its registers
template <class C>
void launch_edge(const Params &P, const StepPtrs &S, int nedge, int ntx, int a_lo, int a_hi, int b_lo, int b_hi,
                 cudaStream_t st) {
  if (nedge <= 0) return;
  if constexpr (C::CPT >= 2) {
    static const int sms = [] {
      int dev = 0, n = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
      return n > 0 ? n : 1;
    }();
    if (nedge <= sms) {
      using H = typename FrameCfg<C, true>::type;
      const int nb = C::CPT * nedge;
      if (P.extrap) step_edge_kernel<C, true, true><<<nb, H::NT, 0, st>>>(P, S, ntx, a_lo, a_hi, b_lo, b_hi);
      else step_edge_kernel<C, false, true><<<nb, H::NT, 0, st>>>(P, S, ntx, a_lo, a_hi, b_lo, b_hi);
      return;
    }
  }
  if (P.extrap) step_edge_kernel<C, true><<<nedge, C::NT, 0, st>>>(P, S, ntx, a_lo, a_hi, b_lo, b_hi);
  else step_edge_kernel<C, false><<<nedge, C::NT, 0, st>>>(P, S, ntx, a_lo, a_hi, b_lo, b_hi);
}

// longest walk (tiles per persistent block) beside which a frame kernel runs
constexpr int kForkWalk = 16;

// With a fork (S.fork) the frame kernel of an iteration runs on the fork's
// side stream beside the interior kernel: both read iteration k and write
// disjoint nodes of k + 1.  fork_begin() records the fork point on `st` and
// returns whether the side stream is used; fork_end() makes `st` wait for it.
inline bool fork_begin(const StepPtrs &S, cudaStream_t st, bool want) {
  if (!S.fork || !want) return false;
  cudaEventRecord(S.fork->fork, st);
  cudaStreamWaitEvent(S.fork->side, S.fork->fork, 0);
  return true;
}

inline void fork_end(const StepPtrs &S, cudaStream_t st, bool on) {
  if (!on) return;
  cudaEventRecord(S.fork->join, S.fork->side);
  cudaStreamWaitEvent(st, S.fork->join, 0);
}

template <class C>
int step_kernel_count(const Params &P) {
  const int ntx = (P.nx + C::TX - 1) / C::TX, nty = (P.ny + C::TY - 1) / C::TY;
  int a_lo, a_hi, b_lo, b_hi;
  interior_range(P.nx, P.ny, C::TX, C::TY, a_lo, a_hi, b_lo, b_hi);
  const int ni = a_hi - a_lo, nj = b_hi - b_lo;
  return (ni > 0 && nj > 0 ? 1 : 0) + (ntx * nty - ni * nj > 0 ? 1 : 0);
}

template <class C>
cudaError_t launch_step(const Params &P, const StepPtrs &S, cudaStream_t st) {
  const int ntx = (P.nx + C::TX - 1) / C::TX, nty = (P.ny + C::TY - 1) / C::TY;
  int a_lo, a_hi, b_lo, b_hi;
  interior_range(P.nx, P.ny, C::TX, C::TY, a_lo, a_hi, b_lo, b_hi);
  const int ni = a_hi - a_lo, nj = b_hi - b_lo;
  const int nedge = ntx * nty - ni * nj;
  const bool beside = fork_begin(S, st, ni > 0 && nj > 0 && nedge > 0);
  if (beside) launch_edge<C>(P, S, nedge, ntx, a_lo, a_hi, b_lo, b_hi, S.fork->side);
  if (ni > 0 && nj > 0) step_interior_kernel<C><<<dim3(ni, nj), C::NT, 0, st>>>(P, S, a_lo, b_lo);
  if (!beside) launch_edge<C>(P, S, nedge, ntx, a_lo, a_hi, b_lo, b_hi, st);
  fork_end(S, st, beside);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ TMA-staged interior tiles
// One 3-D TMA box brings the nine g planes of the tile plus a 3-node halo
// (the streaming sources of the 2-node u halo) into shared memory, one 2-D
// box brings u on the tile plus a 2-node halo; both complete on one mbarrier.
// Streaming then reads shared memory, u(t+dt) is formed in place, and the
// collision re-reads the streamed populations from shared memory.

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const void *tmap, int c0, int c1, int c2, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_addr(dst)),
      "l"((uint64_t)tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int c0, int c1, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"((uint64_t)tmap), "r"(c0), "r"(c1), "r"(smem_addr(bar))
      : "memory");
}

// bound on mbarrier polls (each try_wait also suspends in hardware for a while)
constexpr uint32_t kMaxPolls = 1u << 22;

// (box geometry in lbs_tiles.h: TmaGeom)
template <class C>
struct TmaCfg : TmaGeom<C::TX, C::TY, (int)sizeof(typename C::gs), (int)sizeof(typename C::us)> {
  using B = TmaGeom<C::TX, C::TY, (int)sizeof(typename C::gs), (int)sizeof(typename C::us)>;
  using gs = typename C::gs;
  using us = typename C::us;
  using real = typename C::real;
  static constexpr int TX = C::TX, TY = C::TY, GW = B::GW, GH = B::GH, UW = B::UW, UH = B::UH, XO = B::XO;
  // the u map copies 16-byte records as pairs of 8-byte elements (a raw
  // copy), so a box row holds 2 UW elements: at most 128 records
  static constexpr int UEL = (int)(sizeof(us) / sizeof(real)); // reals per u record (2 or 4)
  static constexpr int UQ = (int)(sizeof(us) / 8);
  static_assert(UQ * UW <= 256, "a TMA box row holds at most 256 elements");
  static constexpr size_t G_BYTES = (size_t)9 * GH * GW * sizeof(gs);
  static constexpr size_t U_BYTES = (size_t)UH * UW * sizeof(us);
  static constexpr size_t N_BYTES = (size_t)4 * (TY + 2) * (TX + 2) * sizeof(real);
  // N on R1 overwrites the u box once every thread has read its taps when it
  // fits there (FP32 and FP16 storage: float N, 16-byte u records); FP64 has
  // its own N array
  static constexpr bool N_IN_U = N_BYTES <= U_BYTES;
  static constexpr size_t OFF_U = (G_BYTES + 127) / 128 * 128;
  static constexpr size_t OFF_N = N_IN_U ? OFF_U : OFF_U + (U_BYTES + 127) / 128 * 128;
  static constexpr size_t OFF_BAR = N_IN_U ? OFF_U + (U_BYTES + 15) / 16 * 16 : OFF_N + (N_BYTES + 15) / 16 * 16;
  static constexpr size_t SMEM = OFF_BAR + 16;
};

// Phases 1-3 of a TMA-staged interior tile at (x0, y0) whose g box (sg) and
// u box (su) have landed: u(t+dt) on R2 in place, N on R1 into snb, then
// streaming from the g box, source, collision and the stores.  With
// TmaCfg::N_IN_U, snb is the u box itself: every thread computes its N
// entries into registers and keeps its own nodes' u for the store, and the
// entries are written once all threads have read their u taps.
template <class C>
__device__ __forceinline__ void tma_tile(const Params &P, const StepPtrs &S, const typename C::gs *sg,
                                         typename C::us *su, typename C::real *snb, int x0, int y0) {
  using T = TmaCfg<C>;
  using R = typename C::real;
  using us = typename C::us;
  using gs = typename C::gs;
  // g is held in units of g * 2^gshift (1 unless FP16 storage)
  const R inv = gscale_inv<gs, R>(P), scl = gscale<gs, R>(P);
  const R kap = (R)P.kappa * inv;
  auto G = [&](int q, int r, int c) -> R {
    const gs v = sg[((size_t)q * T::GH + r) * T::GW + c];
    if constexpr (sizeof(gs) == 2) return __half2float(v);
    else return (R)v;
  };
  // phase 1: u(t+dt) on R2, in place (R2 position (cx, cy) = node (x0-2+cx, y0-2+cy);
  // its g row is cy+1, its g column cx+XO-2)
  for (int e = threadIdx.x; e < T::UW * T::UH; e += C::NT) {
    const int cx = e % T::UW, cy = e / T::UW;
    const int gr = cy + 1, gc = cx + T::XO - 2;
    R p[9], o[9];
#pragma unroll
    for (int q = 1; q < 9; ++q) {
      p[q] = G(q, gr - ey(q), gc - ex(q));
      o[q] = G(q, gr, gc);
    }
    // first moments of own and streamed populations, as gather() forms them
    R gx, gy, fx, fy;
    first_moment(o, gx, gy);
    first_moment(p, fx, fy);
    su[e] = uadd_k(su[e], kap, gx + fx, gy + fy);
  }
  __syncthreads();
  // phase 2: N on R1
  constexpr int W1 = C::TX + 2, H1 = C::TY + 2, NE = W1 * H1, NPER = (NE + C::NT - 1) / C::NT;
  const int tx = threadIdx.x % C::TX, ty = threadIdx.x / C::TX;
  const R hdx = R(0.5) * (R)P.inv_dx;
  // own nodes' u(t+dt), read before N may overwrite the box
  us uown[C::CPT];
#pragma unroll
  for (int i = 0; i < C::CPT; ++i) uown[i] = su[(ty + i * C::NTY + 2) * T::UW + (tx + 2)];
  {
    const R lam = (R)P.lam, mu = (R)P.mu;
    R nreg[T::N_IN_U ? NPER : 1][4];
#pragma unroll
    for (int k = 0; k < NPER; ++k) {
      const int e = threadIdx.x + k * C::NT;
      if (e >= NE) break;
      const int rx = e % W1, ry = e / W1;
      const int c = (ry + 1) * T::UW + (rx + 1);
      R dxx, dxy, dyx, dyy, H[4], N[4];
      udiff(su[c + 1], su[c - 1], dxx, dxy);
      udiff(su[c + T::UW], su[c - T::UW], dyx, dyy);
      H[0] = dxx * hdx;
      H[1] = dyx * hdx;
      H[2] = dxy * hdx;
      H[3] = dyy * hdx;
      material<R>(P, lam, mu, H, N);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        if constexpr (T::N_IN_U) nreg[k][m] = N[m];
        else snb[(m * H1 + ry) * W1 + rx] = N[m];
      }
    }
    if constexpr (T::N_IN_U) {
      __syncthreads();  // every u tap has been read: N may overwrite the box
#pragma unroll
      for (int k = 0; k < NPER; ++k) {
        const int e = threadIdx.x + k * C::NT;
        if (e >= NE) break;
        const int rx = e % W1, ry = e / W1;
#pragma unroll
        for (int m = 0; m < 4; ++m) snb[(m * H1 + ry) * W1 + rx] = nreg[k][m];
      }
    }
  }
  __syncthreads();
  // phase 3: stream again from shared memory, source, collision, store
  const size_t plane = (size_t)P.ny * P.pitch;
  const CollideK<R> K = collide_k<R>((R)P.omega, (R)P.sigma, scl);
  const R sbx = (R)(P.rho0 * P.body[0]), sby = (R)(P.rho0 * P.body[1]);
  gs *__restrict__ go = (gs *)S.g_out;
  us *__restrict__ uo = (us *)S.u_out;
#pragma unroll
  for (int i = 0; i < C::CPT; ++i) {
    const int lx = tx, ly = ty + i * C::NTY;
    const int gr = ly + 3, gc = lx + T::XO;
    R f[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) f[q] = G(q, gr - ey(q), gc - ex(q));
    const int rx = lx + 1, ry = ly + 1;
    auto n = [&](int m, int yy, int xx) -> R { return snb[(m * H1 + yy) * W1 + xx]; };
    const R Sx = fmr(n(0, ry, rx + 1) - n(0, ry, rx - 1), hdx, fmr(n(1, ry + 1, rx) - n(1, ry - 1, rx), hdx, sbx));
    const R Sy = fmr(n(2, ry, rx + 1) - n(2, ry, rx - 1), hdx, fmr(n(3, ry + 1, rx) - n(3, ry - 1, rx), hdx, sby));
    collide<R>(f, Sx, Sy, K);
    const size_t idx = (size_t)(y0 + ly) * P.pitch + (x0 + lx);
#pragma unroll
    for (int q = 0; q < 9; ++q) gstore(go, q * plane + idx, f[q], scl);
    uo[idx] = uown[i];
  }
}

template <class C>
__global__ void __launch_bounds__(C::NT) step_tma_kernel(const Params P, const StepPtrs S,
                                                         const __grid_constant__ CUtensorMap tm_g,
                                                         const __grid_constant__ CUtensorMap tm_u, int a_lo, int b_lo) {
  using T = TmaCfg<C>;
  using R = typename C::real;
  using us = typename C::us;
  using gs = typename C::gs;
  extern __shared__ __align__(128) unsigned char dsm[];
  gs *sg = (gs *)dsm;                      // [9][GH][GW]
  us *su = (us *)(dsm + T::OFF_U);         // [UH][UW]
  R *snb = (R *)(dsm + T::OFF_N);          // [4][TY+2][TX+2]
  uint64_t *bar = (uint64_t *)(dsm + T::OFF_BAR);
  const int x0 = (a_lo + blockIdx.x) * C::TX, y0 = (b_lo + blockIdx.y) * C::TY;

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_expect_tx(bar, (uint32_t)(T::G_BYTES + T::U_BYTES));
    tma_load_3d(sg, &tm_g, x0 - T::XO, y0 - 3, 0, bar);
    tma_load_2d(su, &tm_u, T::UQ * (x0 - 2), y0 - 2, bar);
  }
  __syncthreads();  // the barrier is initialised before anyone polls it
  int ok = 0;
  for (uint32_t i = 0; i < kMaxPolls; ++i)
    if (mbar_try_wait(bar, 0)) {
      ok = 1;
      break;
    }
  if (!__syncthreads_and(ok)) {
    // the copies did not land in time: report and leave without touching
    // the tile (the host turns the flag into LBS_ETIMEOUT)
    if (threadIdx.x == 0 && S.err) atomicExch(S.err, 1);
    return;
  }

  tma_tile<C>(P, S, sg, su, snb, x0, y0);
}

template <class C>
cudaError_t launch_step_tma(const Params &P, const StepPtrs &S, cudaStream_t st) {
  using T = TmaCfg<C>;
  const int ntx = (P.nx + C::TX - 1) / C::TX, nty = (P.ny + C::TY - 1) / C::TY;
  int a_lo, a_hi, b_lo, b_hi;
  interior_range(P.nx, P.ny, C::TX, C::TY, a_lo, a_hi, b_lo, b_hi);
  const int ni = a_hi - a_lo, nj = b_hi - b_lo;
  if (ni > 0 && nj > 0 && (!S.tm_g || !S.tm_u)) return cudaErrorInvalidValue;
  const int nedge = ntx * nty - ni * nj;
  const bool beside = fork_begin(S, st, ni > 0 && nj > 0 && nedge > 0);
  if (beside) launch_edge<C>(P, S, nedge, ntx, a_lo, a_hi, b_lo, b_hi, S.fork->side);
  if (ni > 0 && nj > 0)
    step_tma_kernel<C><<<dim3(ni, nj), C::NT, T::SMEM, st>>>(P, S, *(const CUtensorMap *)S.tm_g,
                                                               *(const CUtensorMap *)S.tm_u, a_lo, b_lo);
  if (!beside) launch_edge<C>(P, S, nedge, ntx, a_lo, a_hi, b_lo, b_hi, st);
  fork_end(S, st, beside);
  return cudaGetLastError();
}

// Persistent variant: each block walks interior tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... with two shared-memory stages, prefetching tile
// t + gridDim.x by TMA while it computes tile t.
template <class C>
struct Tma2Cfg {
  using T = TmaCfg<C>;
  // g and u of one tile (128-aligned); N in the u box of the stage, or in one
  // array after both stages
  static constexpr size_t STAGE = T::OFF_U + (T::U_BYTES + 127) / 128 * 128;
  static constexpr size_t OFF_N = 2 * STAGE;
  static constexpr size_t OFF_BAR = T::N_IN_U ? OFF_N : OFF_N + (T::N_BYTES + 15) / 16 * 16;
  static constexpr size_t SMEM = OFF_BAR + 32;
};

__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <class C>
__device__ __forceinline__ void tma2_issue(unsigned char *stage, uint64_t *bar, const CUtensorMap &tm_g,
                                           const CUtensorMap &tm_u, int x0, int y0) {
  using T = TmaCfg<C>;
  mbar_expect_tx(bar, (uint32_t)(T::G_BYTES + T::U_BYTES));
  tma_load_3d(stage, &tm_g, x0 - T::XO, y0 - 3, 0, bar);
  tma_load_2d(stage + T::OFF_U, &tm_u, T::UQ * (x0 - 2), y0 - 2, bar);
}

template <class C>
__global__ void __launch_bounds__(C::NT) step_tma2_kernel(const Params P, const StepPtrs S,
                                                          const __grid_constant__ CUtensorMap tm_g,
                                                          const __grid_constant__ CUtensorMap tm_u, int a_lo, int b_lo,
                                                          int ni, int ntiles) {
  using T = TmaCfg<C>;
  using T2 = Tma2Cfg<C>;
  using R = typename C::real;
  using us = typename C::us;
  using gs = typename C::gs;
  extern __shared__ __align__(128) unsigned char dsm[];
  uint64_t *bar = (uint64_t *)(dsm + T2::OFF_BAR);  // bar[0], bar[1]
  auto tile_xy = [&](int t, int &x0, int &y0) {
    x0 = (a_lo + t % ni) * C::TX;
    y0 = (b_lo + t / ni) * C::TY;
  };
  int t = blockIdx.x;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    if (t < ntiles) {
      int x0, y0;
      tile_xy(t, x0, y0);
      tma2_issue<C>(dsm, &bar[0], tm_g, tm_u, x0, y0);
    }
  }
  __syncthreads();

  for (int i = 0; t < ntiles; ++i, t += gridDim.x) {
    const int s = i & 1;
    unsigned char *stage = dsm + s * T2::STAGE;
    gs *sg = (gs *)stage;
    us *su = (us *)(stage + T::OFF_U);
    // prefetch the next tile into the other stage (its previous tile is done:
    // the barrier at the end of the last iteration)
    const int tn = t + gridDim.x;
    if (threadIdx.x == 0 && tn < ntiles) {
      int x1, y1;
      tile_xy(tn, x1, y1);
      fence_async_shared();
      tma2_issue<C>(dsm + (s ^ 1) * T2::STAGE, &bar[s ^ 1], tm_g, tm_u, x1, y1);
    }
    int ok = 0;
    const uint32_t parity = (uint32_t)((i >> 1) & 1);
    for (uint32_t it = 0; it < kMaxPolls; ++it)
      if (mbar_try_wait(&bar[s], parity)) {
        ok = 1;
        break;
      }
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) {
        if (S.err) atomicExch(S.err, 1);
        // let the prefetch into the other stage land before leaving
        if (tn < ntiles)
          for (uint32_t it = 0; it < kMaxPolls; ++it)
            if (mbar_try_wait(&bar[s ^ 1], (uint32_t)(((i + 1) >> 1) & 1))) break;
      }
      return;
    }
    int x0, y0;
    tile_xy(t, x0, y0);
    tma_tile<C>(P, S, sg, su, T::N_IN_U ? (R *)su : (R *)(dsm + T2::OFF_N), x0, y0);
    __syncthreads();  // this stage is free for the prefetch after next
  }
}

template <class C>
cudaError_t launch_step_tma2(const Params &P, const StepPtrs &S, cudaStream_t st) {
  using T2 = Tma2Cfg<C>;
  const int ntx = (P.nx + C::TX - 1) / C::TX, nty = (P.ny + C::TY - 1) / C::TY;
  int a_lo, a_hi, b_lo, b_hi;
  interior_range(P.nx, P.ny, C::TX, C::TY, a_lo, a_hi, b_lo, b_hi);
  const int ni = a_hi - a_lo, nj = b_hi - b_lo;
  if (ni > 0 && nj > 0 && (!S.tm_g || !S.tm_u)) return cudaErrorInvalidValue;
  // resident blocks (computed once, after the shared-memory opt-in that
  // selecting the variant made; thread-safe initialisation)
  static const int blocks = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step_tma2_kernel<C>, C::NT, T2::SMEM);
    return (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  }();
  const int ntiles = ni * nj;
  // the frame kernel runs beside the interior one only while the walk is
  // short: beside a long persistent walk it holds back blocks whose tiles are
  // fixed (measured at 16384^2 with FP16 storage, 1150 tiles per block: 33
  // instead of 60 GLUPS; at 4096 x 256, 4 tiles per block: 10 % faster)
  const int nedge = ntx * nty - ni * nj;
  const bool beside = fork_begin(S, st, ni > 0 && nj > 0 && nedge > 0 && ntiles <= kForkWalk * blocks);
  if (beside) launch_edge<C>(P, S, nedge, ntx, a_lo, a_hi, b_lo, b_hi, S.fork->side);
  if (ni > 0 && nj > 0) {
    step_tma2_kernel<C><<<ntiles < blocks ? ntiles : blocks, C::NT, T2::SMEM, st>>>(
        P, S, *(const CUtensorMap *)S.tm_g, *(const CUtensorMap *)S.tm_u, a_lo, b_lo, ni, ntiles);
  }
  if (!beside) launch_edge<C>(P, S, nedge, ntx, a_lo, a_hi, b_lo, b_hi, st);
  fork_end(S, st, beside);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ two iterations per launch
// Temporal blocking on periodic lattices: a block advances its output tile
// by two iterations, k -> k + 2, from g_k on the tile plus 6 nodes and u_k on
// the tile plus 5, both staged in shared memory (Fuse2Geom in lbs_tiles.h).
// First iteration over the enlarged region: u_{k+1} on tile + 5, N on tile
// + 4, g_{k+1} on tile + 3 (rounded to the storage type into a second shared
// g array, exactly as a single iteration stores it); second iteration on the
// tile: u_{k+2} on tile + 2, N on tile + 1, g_{k+2} on the tile.  Each node's
// arithmetic is that of the single-iteration kernels, so two fused
// iterations equal two single ones bitwise.  DRAM traffic per node update is
// half of one iteration's; the halo regions are recomputed (about 1.3x the
// arithmetic).  Interior tiles (tile + 6 inside the lattice) stage by TMA;
// the frame tiles gather their boxes with wrapped loads.
template <class C>
struct Fuse2Cfg : Fuse2Geom<C::TX, C::TY, (int)sizeof(typename C::gs), (int)sizeof(typename C::us)> {
  using B = Fuse2Geom<C::TX, C::TY, (int)sizeof(typename C::gs), (int)sizeof(typename C::us)>;
  using gs = typename C::gs;
  using us = typename C::us;
  using real = typename C::real;
  static constexpr int UEL = (int)(sizeof(us) / sizeof(real));
  static constexpr size_t G_BYTES = (size_t)9 * B::GH * B::GW * sizeof(gs);
  static constexpr size_t U_BYTES = (size_t)B::UH * B::UW * sizeof(us);
  static constexpr size_t H_BYTES = (size_t)9 * B::HH * B::HW * sizeof(gs);
  static constexpr size_t N_BYTES = (size_t)4 * B::NH * B::NW * sizeof(real);
  static constexpr size_t OFF_U = (G_BYTES + 127) / 128 * 128;
  static constexpr size_t OFF_H = OFF_U + (U_BYTES + 127) / 128 * 128;
  static constexpr size_t OFF_N = OFF_H + (H_BYTES + 15) / 16 * 16;
  static constexpr size_t OFF_BAR = OFF_N + (N_BYTES + 15) / 16 * 16;
  static constexpr size_t SMEM = OFF_BAR + 16;
};

template <class G>
__device__ __forceinline__ typename G::real fconv(typename G::gs v) {
  if constexpr (sizeof(typename G::gs) == 2) return __half2float(v);
  else return (typename G::real)v;
}
template <class G>
__device__ __forceinline__ typename G::gs fstore(typename G::real v) {
  if constexpr (sizeof(typename G::gs) == 2) return __float2half_rn(v);
  else return (typename G::gs)v;
}

// both iterations of one tile from its staged boxes; stores the nodes of the
// tile that lie in the lattice
template <class C>
__device__ __forceinline__ void fused2_tile(const Params &P, const StepPtrs &S, const typename C::gs *sg,
                                            typename C::us *su, typename C::gs *sh, typename C::real *sn, int x0,
                                            int y0) {
  using F = Fuse2Cfg<C>;
  using R = typename C::real;
  using us = typename C::us;
  using gs = typename C::gs;
  const R inv = gscale_inv<gs, R>(P), scl = gscale<gs, R>(P);
  const R kap = (R)P.kappa * inv, hdx = R(0.5) * (R)P.inv_dx;
  const R lam = (R)P.lam, mu = (R)P.mu;
  const CollideK<R> K = collide_k<R>((R)P.omega, (R)P.sigma, scl);
  const R sbx = (R)(P.rho0 * P.body[0]), sby = (R)(P.rho0 * P.body[1]);
  // u(t+dt) at node offset (i, j) from the populations of array A (g box or g1)
  auto advance_u = [&](auto A, int i, int j) {
    R p[9], o[9];
#pragma unroll
    for (int q = 1; q < 9; ++q) {
      p[q] = A(q, i - ex(q), j - ey(q));
      o[q] = A(q, i, j);
    }
    R gx, gy, fx, fy;
    first_moment(o, gx, gy);
    first_moment(p, fx, fy);
    us &uu = su[F::u(i, j)];
    uu = uadd_k(uu, kap, gx + fx, gy + fy);
  };
  // N at node offset (i, j) from u in the u box
  auto stress = [&](int i, int j) {
    R dxx, dxy, dyx, dyy, H[4], N[4];
    udiff(su[F::u(i + 1, j)], su[F::u(i - 1, j)], dxx, dxy);
    udiff(su[F::u(i, j + 1)], su[F::u(i, j - 1)], dyx, dyy);
    H[0] = dxx * hdx;
    H[1] = dyx * hdx;
    H[2] = dxy * hdx;
    H[3] = dyy * hdx;
    material<R>(P, lam, mu, H, N);
#pragma unroll
    for (int m = 0; m < 4; ++m) sn[F::n(m, i, j)] = N[m];
  };
  // streamed populations of node (i, j) from array A, collided with S = div N
  auto collide_at = [&](auto A, int i, int j, R f[9]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) f[q] = A(q, i - ex(q), j - ey(q));
    auto n = [&](int m, int ii, int jj) -> R { return sn[F::n(m, ii, jj)]; };
    const R Sx = fmr(n(0, i + 1, j) - n(0, i - 1, j), hdx, fmr(n(1, i, j + 1) - n(1, i, j - 1), hdx, sbx));
    const R Sy = fmr(n(2, i + 1, j) - n(2, i - 1, j), hdx, fmr(n(3, i, j + 1) - n(3, i, j - 1), hdx, sby));
    collide<R>(f, Sx, Sy, K);
  };
  auto Gk = [&](int q, int i, int j) -> R { return fconv<F>(sg[F::g(q, i, j)]); };
  auto G1 = [&](int q, int i, int j) -> R { return fconv<F>(sh[F::h(q, i, j)]); };

  // first iteration: u_{k+1} on tile + 5, N on tile + 4, g_{k+1} on tile + 3
  for (int e = threadIdx.x; e < F::UW * F::UH; e += C::NT) advance_u(Gk, e % F::UW - 5, e / F::UW - 5);
  __syncthreads();
  for (int e = threadIdx.x; e < F::NW * F::NH; e += C::NT) stress(e % F::NW - 4, e / F::NW - 4);
  __syncthreads();
  for (int e = threadIdx.x; e < F::HW * F::HH; e += C::NT) {
    const int i = e % F::HW - 3, j = e / F::HW - 3;
    R f[9];
    collide_at(Gk, i, j, f);
#pragma unroll
    for (int q = 0; q < 9; ++q) sh[F::h(q, i, j)] = fstore<F>(f[q]);
  }
  __syncthreads();
  // second iteration: u_{k+2} on tile + 2, N on tile + 1, g_{k+2} on the tile
  constexpr int W2 = C::TX + 4, W1 = C::TX + 2;
  for (int e = threadIdx.x; e < W2 * (C::TY + 4); e += C::NT) advance_u(G1, e % W2 - 2, e / W2 - 2);
  __syncthreads();
  for (int e = threadIdx.x; e < W1 * (C::TY + 2); e += C::NT) stress(e % W1 - 1, e / W1 - 1);
  __syncthreads();
  const size_t plane = (size_t)P.ny * P.pitch;
  gs *__restrict__ go = (gs *)S.g_out;
  us *__restrict__ uo = (us *)S.u_out;
  const int tx = threadIdx.x % C::TX, ty = threadIdx.x / C::TX;
#pragma unroll
  for (int c = 0; c < C::CPT; ++c) {
    const int i = tx, j = ty + c * C::NTY;
    R f[9];
    collide_at(G1, i, j, f);
    const int x = x0 + i, y = y0 + j;
    if (x >= P.nx || y >= P.ny) continue;
    const size_t idx = (size_t)y * P.pitch + x;
#pragma unroll
    for (int q = 0; q < 9; ++q) gstore(go, q * plane + idx, f[q], scl);
    uo[idx] = su[F::u(i, j)];
  }
}

template <class C>
__global__ void __launch_bounds__(C::NT) step_fused2_tma_kernel(const Params P, const StepPtrs S,
                                                                const __grid_constant__ CUtensorMap tm_g,
                                                                const __grid_constant__ CUtensorMap tm_u, int a_lo,
                                                                int b_lo) {
  using F = Fuse2Cfg<C>;
  using gs = typename C::gs;
  using us = typename C::us;
  using R = typename C::real;
  extern __shared__ __align__(128) unsigned char dsm[];
  gs *sg = (gs *)dsm;
  us *su = (us *)(dsm + F::OFF_U);
  gs *sh = (gs *)(dsm + F::OFF_H);
  R *sn = (R *)(dsm + F::OFF_N);
  uint64_t *bar = (uint64_t *)(dsm + F::OFF_BAR);
  const int x0 = (a_lo + blockIdx.x) * C::TX, y0 = (b_lo + blockIdx.y) * C::TY;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_expect_tx(bar, (uint32_t)(F::G_BYTES + F::U_BYTES));
    tma_load_3d(sg, &tm_g, x0 - F::XO, y0 - 6, 0, bar);
    tma_load_2d(su, &tm_u, F::UEL * (x0 - 5), y0 - 5, bar);
  }
  __syncthreads();  // the barrier is initialised before anyone polls it
  int ok = 0;
  for (uint32_t i = 0; i < kMaxPolls; ++i)
    if (mbar_try_wait(bar, 0)) {
      ok = 1;
      break;
    }
  if (!__syncthreads_and(ok)) {
    if (threadIdx.x == 0 && S.err) atomicExch(S.err, 1);
    return;
  }
  fused2_tile<C>(P, S, sg, su, sh, sn, x0, y0);
}

// frame tiles of a periodic lattice: the boxes gathered with wrapped loads
template <class C>
__global__ void __launch_bounds__(C::NT) step_fused2_edge_kernel(const Params P, const StepPtrs S, int ntx, int a_lo,
                                                                 int a_hi, int b_lo, int b_hi) {
  using F = Fuse2Cfg<C>;
  using gs = typename C::gs;
  using us = typename C::us;
  using R = typename C::real;
  extern __shared__ __align__(128) unsigned char dsm[];
  gs *sg = (gs *)dsm;
  us *su = (us *)(dsm + F::OFF_U);
  gs *sh = (gs *)(dsm + F::OFF_H);
  R *sn = (R *)(dsm + F::OFF_N);
  int a, b;
  edge_tile(blockIdx.x, ntx, a_lo, a_hi, b_lo, b_hi, a, b);
  const int x0 = a * C::TX, y0 = b * C::TY;
  const gs *__restrict__ g = (const gs *)S.g_in;
  const us *__restrict__ u = (const us *)S.u_in;
  const size_t plane = (size_t)P.ny * P.pitch;
  // the used columns of the g box: node offsets -6 .. TX + 5
  constexpr int GU = C::TX + 12;
  for (int e = threadIdx.x; e < 9 * F::GH * GU; e += C::NT) {
    const int q = e / (F::GH * GU), r = e % (F::GH * GU);
    const int i = r % GU - 6, j = r / GU - 6;
    int x = x0 + i, y = y0 + j;
    locate(P, x, y);
    sg[F::g(q, i, j)] = g[q * plane + (size_t)y * P.pitch + x];
  }
  for (int e = threadIdx.x; e < F::UW * F::UH; e += C::NT) {
    const int i = e % F::UW - 5, j = e / F::UW - 5;
    int x = x0 + i, y = y0 + j;
    locate(P, x, y);
    su[e] = u[(size_t)y * P.pitch + x];
  }
  __syncthreads();
  fused2_tile<C>(P, S, sg, su, sh, sn, x0, y0);
}

// Fused iterations apply to lattices with every edge periodic and both sides
// at least 16 nodes (a tile's read region then wraps at most once); other
// lattices advance one iteration per call.
inline bool fused2_applies(const Params &P) { return P.per_x && P.per_y && P.nx >= 16 && P.ny >= 16; }

template <class C>
cudaError_t launch_step_fused2(const Params &P, const StepPtrs &S, cudaStream_t st) {
  using F = Fuse2Cfg<C>;
  const int ntx = (P.nx + C::TX - 1) / C::TX, nty = (P.ny + C::TY - 1) / C::TY;
  int a_lo, a_hi, b_lo, b_hi;
  interior_range_m(P.nx, P.ny, C::TX, C::TY, 6, a_lo, a_hi, b_lo, b_hi);
  const int ni = a_hi - a_lo, nj = b_hi - b_lo;
  if (ni > 0 && nj > 0 && (!S.tm_g || !S.tm_u)) return cudaErrorInvalidValue;
  const int nedge = ntx * nty - ni * nj;
  const bool beside = fork_begin(S, st, ni > 0 && nj > 0 && nedge > 0);
  cudaStream_t es = beside ? S.fork->side : st;
  if (nedge > 0) step_fused2_edge_kernel<C><<<nedge, C::NT, F::SMEM, es>>>(P, S, ntx, a_lo, a_hi, b_lo, b_hi);
  if (ni > 0 && nj > 0)
    step_fused2_tma_kernel<C><<<dim3(ni, nj), C::NT, F::SMEM, st>>>(P, S, *(const CUtensorMap *)S.tm_g,
                                                                      *(const CUtensorMap *)S.tm_u, a_lo, b_lo);
  fork_end(S, st, beside);
  return cudaGetLastError();
}

template <class C>
bool make_fused2_maps(const Params &P, const void *g, const void *u, void *out_g, void *out_u) {
  using F = Fuse2Cfg<C>;
  using gs = typename C::gs;
  using R = typename C::real;
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }();
  if (!encode) return false;
  const CUtensorMapDataType gt = sizeof(gs) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                 : sizeof(gs) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const cuuint64_t gdim[3] = {(cuuint64_t)P.pitch, (cuuint64_t)P.ny, 9};
  const cuuint64_t gstr[2] = {(cuuint64_t)P.pitch * sizeof(gs), (cuuint64_t)P.ny * P.pitch * sizeof(gs)};
  const cuuint32_t gbox[3] = {(cuuint32_t)F::GW, (cuuint32_t)F::GH, 9};
  const cuuint32_t est[3] = {1, 1, 1};
  CUresult r1 = encode((CUtensorMap *)out_g, gt, 3, const_cast<void *>(g), gdim, gstr, gbox, est,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  const CUtensorMapDataType ut = sizeof(R) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const cuuint64_t udim[2] = {(cuuint64_t)F::UEL * P.pitch, (cuuint64_t)P.ny};
  const cuuint64_t ustr[1] = {(cuuint64_t)F::UEL * P.pitch * sizeof(R)};
  const cuuint32_t ubox[2] = {(cuuint32_t)(F::UEL * F::UW), (cuuint32_t)F::UH};
  CUresult r2 = encode((CUtensorMap *)out_u, ut, 2, const_cast<void *>(u), udim, ustr, ubox, est,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) return false;
  return cudaFuncSetAttribute(step_fused2_tma_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F::SMEM) ==
             cudaSuccess &&
         cudaFuncSetAttribute(step_fused2_edge_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)F::SMEM) == cudaSuccess;
}

// ------------------------------------------------------------------ row-marching strips
// A block owns one TX-wide column of interior tiles over a segment of SH rows
// and marches up it RB rows at a time, one thread per output node of a step.
// Ring buffers in shared memory hold the g rows (nine planes each), u rows and
// N rows still needed; each step loads only its RB new g rows and RB new u
// rows (one TMA row copy each, issued D steps ahead), so the halo is
// recomputed only across x.  Step j (output rows [y, y+RB)): u(t+dt) for rows
// [y+2, y+RB+2), N for rows [y+1, y+RB+1), then streaming, source, collision
// and stores for rows [y, y+RB).
template <class C, int RB_, int SH_, int D_>
struct MarchCfg {
  using T = TmaCfg<C>;
  using gs = typename C::gs;
  using us = typename C::us;
  using real = typename C::real;
  static constexpr int TX = C::TX, RB = RB_, SH = SH_, D = D_, NT = RB * TX;
  static constexpr int GW = T::GW, XO = T::XO, UW = T::UW, W1 = TX + 2, UEL = T::UEL;
  static constexpr int CG = 32, CU = 32, CN = 16;  // ring sizes (rows), powers of two
  // rows in use at step j plus the rows of the D steps in flight
  static_assert(CG >= (D + 1) * RB + 4 && CU >= (D + 1) * RB + 2 && CN >= RB + 2, "rings too small");
  static_assert(SH % RB == 0 && C::TY % RB == 0, "segments split into whole steps");
  static_assert(NT <= 1024 && NT % 32 == 0, "one thread per output node of a step");
  static constexpr size_t G_ROW = (size_t)9 * GW * sizeof(gs);  // bytes one row copy delivers
  static constexpr size_t U_ROW = (size_t)UW * sizeof(us);
  // ring slots start on 128-byte boundaries (the shared-memory alignment of a
  // tensor copy's destination)
  static constexpr size_t G_SLOT = (G_ROW + 127) / 128 * 128;
  static constexpr size_t U_SLOT = (U_ROW + 127) / 128 * 128;
  static_assert(G_SLOT % sizeof(gs) == 0 && U_SLOT % sizeof(us) == 0, "slot strides in elements");
  static constexpr size_t OFF_U = (size_t)CG * G_SLOT;
  static constexpr size_t OFF_N = OFF_U + (size_t)CU * U_SLOT;
  static constexpr size_t OFF_BAR = OFF_N + ((size_t)CN * 4 * W1 * sizeof(real) + 15) / 16 * 16;
  static constexpr size_t SMEM = OFF_BAR + 8 * (D + 1);  // bar[0..D-1]: steps, bar[D]: prologue
};

template <class M>
__device__ __forceinline__ void march_issue(unsigned char *dsm, uint64_t *bar, const CUtensorMap &tm_g,
                                            const CUtensorMap &tm_u, int x0, int g_lo, int ng, int gbase, int u_lo,
                                            int nu, int ubase) {
  mbar_expect_tx(bar, (uint32_t)(ng * M::G_ROW + nu * M::U_ROW));
  for (int r = g_lo; r < g_lo + ng; ++r)
    tma_load_3d(dsm + (size_t)((r - gbase) & (M::CG - 1)) * M::G_SLOT, &tm_g, x0 - M::XO, r, 0, bar);
  for (int r = u_lo; r < u_lo + nu; ++r)
    tma_load_2d(dsm + M::OFF_U + (size_t)((r - ubase) & (M::CU - 1)) * M::U_SLOT, &tm_u, M::UEL * (x0 - 2), r, bar);
}

__device__ __forceinline__ bool march_wait(uint64_t *bar, uint32_t parity) {
  int ok = 0;
  for (uint32_t it = 0; it < kMaxPolls; ++it)
    if (mbar_try_wait(bar, parity)) {
      ok = 1;
      break;
    }
  return __syncthreads_and(ok) != 0;
}

template <class C, class M>
__global__ void __launch_bounds__(M::NT) step_march_kernel(const Params P, const StepPtrs S,
                                                           const __grid_constant__ CUtensorMap tm_g,
                                                           const __grid_constant__ CUtensorMap tm_u, int a_lo, int ni,
                                                           int y_first, int y_last) {
  using R = typename C::real;
  using us = typename C::us;
  using gs = typename C::gs;
  constexpr int RB = M::RB, D = M::D, NT = M::NT, CG = M::CG, CU = M::CU, CN = M::CN, GW = M::GW, UW = M::UW,
                W1 = M::W1;
  extern __shared__ __align__(128) unsigned char dsm[];
  const gs *gr = (const gs *)dsm;             // [CG] slots of [9][GW]
  us *ur = (us *)(dsm + M::OFF_U);            // [CU] slots of [UW]
  R *nr = (R *)(dsm + M::OFF_N);              // [CN][4][W1]
  uint64_t *bar = (uint64_t *)(dsm + M::OFF_BAR);
  const int x0 = (a_lo + (int)(blockIdx.x % ni)) * C::TX;
  const int ys = y_first + (int)(blockIdx.x / ni) * M::SH;
  const int ye = min(ys + M::SH, y_last);
  const int nsteps = (ye - ys) / RB;
  const int gbase = ys - 3, ubase = ys - 2, nbase = ys - 1;
  auto G = [&](int q, int row, int c) -> R {
    const gs v = gr[(size_t)((row - gbase) & (CG - 1)) * (M::G_SLOT / sizeof(gs)) + q * GW + c];
    if constexpr (sizeof(gs) == 2) return __half2float(v);
    else return (R)v;
  };
  auto U = [&](int row, int cx) -> us & { return ur[(size_t)((row - ubase) & (CU - 1)) * (M::U_SLOT / sizeof(us)) + cx]; };
  auto N = [&](int m, int row, int rx) -> R & { return nr[((size_t)((row - nbase) & (CN - 1)) * 4 + m) * W1 + rx]; };
  // the rows step j needs that no earlier copy brought: g [y+3, y+RB+3), u [y+2, y+RB+2)
  auto issue_step = [&](int j) {
    const int y = ys + j * RB;
    march_issue<M>(dsm, &bar[j % D], tm_g, tm_u, x0, y + 3, RB, gbase, y + 2, RB, ubase);
  };

  const R inv = gscale_inv<gs, R>(P), scl = gscale<gs, R>(P);
  const R kap = (R)P.kappa * inv, hdx = R(0.5) * (R)P.inv_dx;
  const R lam = (R)P.lam, mu = (R)P.mu;
  const CollideK<R> K = collide_k<R>((R)P.omega, (R)P.sigma, scl);
  const R sbx = (R)(P.rho0 * P.body[0]), sby = (R)(P.rho0 * P.body[1]);
  const size_t plane = (size_t)P.ny * P.pitch;
  gs *__restrict__ go = (gs *)S.g_out;
  us *__restrict__ uo = (us *)S.u_out;

  // u(t+dt) in place for rows [r0, r0 + nrow) (x: x0-2 .. x0+TX+1)
  auto phase_u = [&](int r0, int nrow) {
    for (int e = threadIdx.x; e < nrow * UW; e += NT) {
      const int row = r0 + e / UW, cx = e % UW, gc = cx + M::XO - 2;
      R p[9], o[9];
#pragma unroll
      for (int q = 1; q < 9; ++q) {
        p[q] = G(q, row - ey(q), gc - ex(q));
        o[q] = G(q, row, gc);
      }
      R gx, gy, fx, fy;
      first_moment(o, gx, gy);
      first_moment(p, fx, fy);
      us &uu = U(row, cx);
      uu = uadd_k(uu, kap, gx + fx, gy + fy);
    }
  };
  // N for rows [r0, r0 + nrow) (x: x0-1 .. x0+TX)
  auto phase_n2 = [&](int r0, int nrow) {
    for (int e = threadIdx.x; e < nrow * W1; e += NT) {
      const int row = r0 + e / W1, rx = e % W1, cx = rx + 1;
      R dxx, dxy, dyx, dyy, H[4], Nn[4];
      udiff(U(row, cx + 1), U(row, cx - 1), dxx, dxy);
      udiff(U(row + 1, cx), U(row - 1, cx), dyx, dyy);
      H[0] = dxx * hdx;
      H[1] = dyx * hdx;
      H[2] = dxy * hdx;
      H[3] = dyy * hdx;
      material<R>(P, lam, mu, H, Nn);
#pragma unroll
      for (int m = 0; m < 4; ++m) N(m, row, rx) = Nn[m];
    }
  };

  // prologue: the warm-up rows (bar[D]) and the first D steps' rows
  if (threadIdx.x == 0) {
    for (int b = 0; b <= D; ++b) mbar_init(&bar[b], 1);
    march_issue<M>(dsm, &bar[D], tm_g, tm_u, x0, ys - 3, 6, gbase, ys - 2, 4, ubase);
    for (int j = 0; j < D && j < nsteps; ++j) issue_step(j);
  }
  __syncthreads();
  if (!march_wait(&bar[D], 0)) {
    // let the copies in flight land before the block leaves
    if (threadIdx.x == 0) {
      if (S.err) atomicExch(S.err, 1);
      for (int j = 0; j < D && j < nsteps; ++j)
        for (uint32_t it = 0; it < kMaxPolls; ++it)
          if (mbar_try_wait(&bar[j], 0)) break;
    }
    return;
  }
  phase_u(ys - 2, 4);
  __syncthreads();
  phase_n2(ys - 1, 2);
  // (the barrier at the top of the first step orders these before their use)

  const int lx = threadIdx.x % C::TX, ly = threadIdx.x / C::TX, rx = lx + 1, gc = lx + M::XO;
  for (int j = 0; j < nsteps; ++j) {
    const int y = ys + j * RB;
    // this step's rows arrived?  (bar[j % D] completes once per D steps)
    if (!march_wait(&bar[j % D], (uint32_t)((j / D) & 1))) {
      if (threadIdx.x == 0) {
        if (S.err) atomicExch(S.err, 1);
        for (int i = j + 1; i < j + D && i < nsteps; ++i)
          for (uint32_t it = 0; it < kMaxPolls; ++it)
            if (mbar_try_wait(&bar[i % D], (uint32_t)((i / D) & 1))) break;
      }
      return;
    }
    // prefetch step j + D into slots of rows no longer needed (the reads of
    // those slots ended before the barrier that closed step j - 1)
    if (threadIdx.x == 0 && j + D < nsteps) {
      fence_async_shared();
      issue_step(j + D);
    }
    phase_u(y + 2, RB);
    __syncthreads();
    phase_n2(y + 1, RB);
    __syncthreads();
    // output node (x0 + lx, y + ly)
    {
      const int row = y + ly;
      R f[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) f[q] = G(q, row - ey(q), gc - ex(q));
      const R Sx = fmr(N(0, row, rx + 1) - N(0, row, rx - 1), hdx, fmr(N(1, row + 1, rx) - N(1, row - 1, rx), hdx, sbx));
      const R Sy = fmr(N(2, row, rx + 1) - N(2, row, rx - 1), hdx, fmr(N(3, row + 1, rx) - N(3, row - 1, rx), hdx, sby));
      collide<R>(f, Sx, Sy, K);
      const size_t idx = (size_t)row * P.pitch + (x0 + lx);
#pragma unroll
      for (int q = 0; q < 9; ++q) gstore(go, q * plane + idx, f[q], scl);
      uo[idx] = U(row, lx + 2);
    }
    __syncthreads();
  }
}

template <class C, class M>
cudaError_t launch_step_march(const Params &P, const StepPtrs &S, cudaStream_t st) {
  const int ntx = (P.nx + C::TX - 1) / C::TX, nty = (P.ny + C::TY - 1) / C::TY;
  int a_lo, a_hi, b_lo, b_hi;
  interior_range(P.nx, P.ny, C::TX, C::TY, a_lo, a_hi, b_lo, b_hi);
  const int ni = a_hi - a_lo, nj = b_hi - b_lo;
  if (ni > 0 && nj > 0 && (!S.tm_g || !S.tm_u)) return cudaErrorInvalidValue;
  const int nedge = ntx * nty - ni * nj;
  const bool beside = fork_begin(S, st, ni > 0 && nj > 0 && nedge > 0);
  if (beside) launch_edge<C>(P, S, nedge, ntx, a_lo, a_hi, b_lo, b_hi, S.fork->side);
  if (ni > 0 && nj > 0) {
    const int y_first = b_lo * C::TY, y_last = b_hi * C::TY;
    const int nseg = (y_last - y_first + M::SH - 1) / M::SH;
    step_march_kernel<C, M><<<ni * nseg, M::NT, M::SMEM, st>>>(P, S, *(const CUtensorMap *)S.tm_g,
                                                               *(const CUtensorMap *)S.tm_u, a_lo, ni, y_first, y_last);
  }
  if (!beside) launch_edge<C>(P, S, nedge, ntx, a_lo, a_hi, b_lo, b_hi, st);
  fork_end(S, st, beside);
  return cudaGetLastError();
}

// row-box TMA descriptors (one g row with its nine planes; one u row)
template <class C, class M>
bool make_march_maps(const Params &P, const void *g, const void *u, void *out_g, void *out_u) {
  using gs = typename C::gs;
  using R = typename C::real;
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return false;
  auto encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  const CUtensorMapDataType gt = sizeof(gs) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                 : sizeof(gs) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const cuuint64_t gdim[3] = {(cuuint64_t)P.pitch, (cuuint64_t)P.ny, 9};
  const cuuint64_t gstr[2] = {(cuuint64_t)P.pitch * sizeof(gs), (cuuint64_t)P.ny * P.pitch * sizeof(gs)};
  const cuuint32_t gbox[3] = {(cuuint32_t)M::GW, 1, 9};
  const cuuint32_t est[3] = {1, 1, 1};
  CUresult r1 = encode((CUtensorMap *)out_g, gt, 3, const_cast<void *>(g), gdim, gstr, gbox, est,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  const CUtensorMapDataType ut = sizeof(R) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const cuuint64_t udim[2] = {(cuuint64_t)M::UEL * P.pitch, (cuuint64_t)P.ny};
  const cuuint64_t ustr[1] = {(cuuint64_t)M::UEL * P.pitch * sizeof(R)};
  const cuuint32_t ubox[2] = {(cuuint32_t)(M::UEL * M::UW), 1};
  CUresult r2 = encode((CUtensorMap *)out_u, ut, 2, const_cast<void *>(u), udim, ustr, ubox, est,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) return false;
  return cudaFuncSetAttribute(step_march_kernel<C, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)M::SMEM) ==
         cudaSuccess;
}

// TMA descriptors for one (g, u) buffer pair and the kernel's shared-memory
// opt-in (host side; called when a handle selects a TMA tile variant)
template <class C>
bool make_tma_maps(const Params &P, const void *g, const void *u, void *out_g, void *out_u) {
  using T = TmaCfg<C>;
  using gs = typename C::gs;
  using R = typename C::real;
  // the driver's tensor-map encoder, looked up once (thread-safe initialisation)
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }();
  if (!encode) return false;
  const CUtensorMapDataType gt = sizeof(gs) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                 : sizeof(gs) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const cuuint64_t gdim[3] = {(cuuint64_t)P.pitch, (cuuint64_t)P.ny, 9};
  const cuuint64_t gstr[2] = {(cuuint64_t)P.pitch * sizeof(gs), (cuuint64_t)P.ny * P.pitch * sizeof(gs)};
  const cuuint32_t gbox[3] = {(cuuint32_t)T::GW, (cuuint32_t)T::GH, 9};
  const cuuint32_t est[3] = {1, 1, 1};
  CUresult r1 = encode((CUtensorMap *)out_g, gt, 3, const_cast<void *>(g), gdim, gstr, gbox, est,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  const cuuint64_t udim[2] = {(cuuint64_t)T::UQ * P.pitch, (cuuint64_t)P.ny};
  const cuuint64_t ustr[1] = {(cuuint64_t)T::UQ * P.pitch * 8};
  const cuuint32_t ubox[2] = {(cuuint32_t)(T::UQ * T::UW), (cuuint32_t)T::UH};
  CUresult r2 = encode((CUtensorMap *)out_u, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(u), udim, ustr, ubox, est,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) return false;
  return cudaFuncSetAttribute(step_tma_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM) ==
             cudaSuccess &&
         cudaFuncSetAttribute(step_tma2_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Tma2Cfg<C>::SMEM) == cudaSuccess;
}

// ------------------------------------------------------------------ init / fields
// u from a double field into the R2 tile (wrap or skip outside)
template <class C>
__device__ void load_r2_from_double(typename C::Smem &sm, const Params &P, const double *u0, int x0, int y0) {
  for (int e = threadIdx.x; e < C::R2W * C::R2H; e += C::NT) {
    const int rx = e % C::R2W, ry = e / C::R2W;
    int x = x0 - 2 + rx, y = y0 - 2 + ry;
    if (!locate(P, x, y)) continue;
    const size_t i = (size_t)y * P.nx + x;
    u_make(u0 ? u0[2 * i] : 0.0, u0 ? u0[2 * i + 1] : 0.0, sm.u[ry][rx]);
  }
}

template <class C>
__device__ void load_r2_from_state(typename C::Smem &sm, const Params &P, const typename C::us *u, int x0, int y0) {
  for (int e = threadIdx.x; e < C::R2W * C::R2H; e += C::NT) {
    const int rx = e % C::R2W, ry = e / C::R2W;
    int x = x0 - 2 + rx, y = y0 - 2 + ry;
    if (!locate(P, x, y)) continue;
    sm.u[ry][rx] = u[(size_t)y * P.pitch + x];
  }
}

// Alg. 1 "Initialise": r0 = -rho0 tr H0, Pi0 = Pi(H0), f0 = feq(r0, rho0 v0 - dt/2 S0, Pi0),
// then the first collision (with S0) gives the stored g.
template <class C>
__global__ void __launch_bounds__(C::NT) init_kernel(const Params P, typename C::gs *g, typename C::us *u,
                                                     typename C::real *bnd, const double *u0, const double *v0) {
  using R = typename C::real;
  __shared__ typename C::Smem sm;
  const int x0 = blockIdx.x * C::TX, y0 = blockIdx.y * C::TY;
  load_r2_from_double<C>(sm, P, u0, x0, y0);
  __syncthreads();
  phase_n<C, true, true>(sm, P, x0, y0, bnd);
  __syncthreads();
  const size_t plane = (size_t)P.ny * P.pitch;
  const R idx_ = (R)P.inv_dx, scl = gscale<typename C::gs, R>(P);
  const int tx = threadIdx.x % C::TX, ty = threadIdx.x / C::TX;
  for (int i = 0; i < C::CPT; ++i) {
    const int lx = tx, ly = ty + i * C::NTY, x = x0 + lx, y = y0 + ly;
    if (x >= P.nx || y >= P.ny) continue;
    R Sx, Sy, H[4];
    Fd<C, true>::div(sm, P, lx + 1, ly + 1, x, y, idx_, (R)(P.rho0 * P.body[0]), (R)(P.rho0 * P.body[1]), Sx, Sy);
    Fd<C, true>::grad(sm, P, lx + 1, ly + 1, x, y, idx_, H);
    const size_t i0 = (size_t)y * P.nx + x;
    const R trH = H[0] + H[3];
    const R r0 = -(R)P.rho0 * trH;
    // A0 = Pi(H0) / cs^2 = -rho0 (H + H^T + tr H I)
    const R rho0 = (R)P.rho0;
    const R Axx = -rho0 * (R(2) * H[0] + trH), Ayy = -rho0 * (R(2) * H[3] + trH), Axy = -rho0 * (H[1] + H[2]);
    const R cr = (R)(P.c * P.inv_cs2 * P.rho0), hs = R(0.5) * (R)P.sigma;
    const R jx = cr * (R)(v0 ? v0[2 * i0] : 0.0) - hs * Sx;
    const R jy = cr * (R)(v0 ? v0[2 * i0 + 1] : 0.0) - hs * Sy;
    R f[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const int e2 = ex(q) * ex(q) + ey(q) * ey(q);
      const R rq = (e2 == 0) ? R(2) * r0 : ((e2 == 1) ? R(0.5) * r0 : -r0);
      const R eAe = R(ex(q) * ex(q)) * Axx + R(2 * ex(q) * ey(q)) * Axy + R(ey(q) * ey(q)) * Ayy;
      f[q] = wq<R>(q) * (rq + R(ex(q)) * jx + R(ey(q)) * jy + R(1.5) * eAe - R(0.5) * (Axx + Ayy)) * scl;
    }
    collide<R>(f, Sx, Sy, collide_k<R>((R)P.omega, (R)P.sigma, scl));
    const size_t idx = (size_t)y * P.pitch + x;
    for (int q = 0; q < 9; ++q) gstore(g, q * plane + idx, f[q], scl);
    u[idx] = sm.u[ly + 2][lx + 2];
  }
}

// Field output of node (x, y) at tile position (lx, ly), into element o of
// the dense arrays: u; v = (c sum e g - dt/2 S) / rho0 (Sect. 3.2: j = rho0 v
// with the half-step source); P = N - Pi(H) (Eq. source).  cr = c / rho0 and
// hr = dt / (2 rho0) are formed once per thread by the caller, so that no
// node divides in FP64.
template <class C>
__device__ __forceinline__ void node_fields(const typename C::Smem &sm, const Params &P, const typename C::gs *g,
                                            size_t plane, size_t idx, int lx, int ly, int x, int y, size_t o,
                                            double cr, double hr, double *uo, double *vo, double *Po) {
  using R = typename C::real;
  const R idx_ = (R)P.inv_dx;
  if (uo) {
    const double2 uv = u_value(sm.u[ly + 2][lx + 2]);
    uo[2 * o] = uv.x;
    uo[2 * o + 1] = uv.y;
  }
  if (vo) {
    R Sx, Sy;
    Fd<C, true>::div(sm, P, lx + 1, ly + 1, x, y, idx_, (R)(P.rho0 * P.body[0]), (R)(P.rho0 * P.body[1]), Sx, Sy);
    // g is held in units of g * 2^gshift (1 unless FP16 storage)
    const R inv = gscale_inv<typename C::gs, R>(P);
    R gq[9], m1x, m1y;
    for (int q = 1; q < 9; ++q) gq[q] = gload(g, q * plane + idx, inv);
    first_moment(gq, m1x, m1y);
    vo[2 * o] = fma(cr, (double)(m1x * inv), -(hr * (double)Sx));
    vo[2 * o + 1] = fma(cr, (double)(m1y * inv), -(hr * (double)Sy));
  }
  if (Po) {
    const R mu = (R)P.mu;
    R H[4];
    Fd<C, true>::grad(sm, P, lx + 1, ly + 1, x, y, idx_, H);
    const R trH = H[0] + H[3];
    Po[4 * o + 0] = (double)(sm.n[0][ly + 1][lx + 1] + mu * (R(2) * H[0] + trH));
    Po[4 * o + 1] = (double)(sm.n[1][ly + 1][lx + 1] + mu * (H[1] + H[2]));
    Po[4 * o + 2] = (double)(sm.n[2][ly + 1][lx + 1] + mu * (H[1] + H[2]));
    Po[4 * o + 3] = (double)(sm.n[3][ly + 1][lx + 1] + mu * (R(2) * H[3] + trH));
  }
}

// u, v and P at every node (x fastest); N on the tile + 1 only when v or P is
// asked for
template <class C>
__global__ void __launch_bounds__(C::NT) fields_kernel(const Params P, const typename C::gs *g, const typename C::us *u,
                                                       double *uo, double *vo, double *Po) {
  using R = typename C::real;
  __shared__ typename C::Smem sm;
  const int x0 = blockIdx.x * C::TX, y0 = blockIdx.y * C::TY;
  load_r2_from_state<C>(sm, P, u, x0, y0);
  __syncthreads();
  if (vo || Po) {
    phase_n<C, true>(sm, P, x0, y0, (R *)nullptr);
    __syncthreads();
  }
  const size_t plane = (size_t)P.ny * P.pitch;
  const double cr = P.c / P.rho0, hr = (0.5 * P.dt) / P.rho0;
  const int tx = threadIdx.x % C::TX, ty = threadIdx.x / C::TX;
  for (int i = 0; i < C::CPT; ++i) {
    const int lx = tx, ly = ty + i * C::NTY, x = x0 + lx, y = y0 + ly;
    if (x >= P.nx || y >= P.ny) continue;
    node_fields<C>(sm, P, g, plane, (size_t)y * P.pitch + x, lx, ly, x, y, (size_t)y * P.nx + x, cr, hr, uo, vo,
                   Po);
  }
}

// ------------------------------------------------------------------ monitors
// per-block partials of: non-finite count, max |u_a|, sum c e g (x, y),
// sum g; a warp shuffle then a shared-memory pass inside each block, and a
// fixed-order final pass (deterministic)
constexpr int kMonThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <class C>
__global__ void __launch_bounds__(kMonThreads) monitor_kernel(const Params P, const typename C::gs *g,
                                                              const typename C::us *u, double *partials) {
  using R = typename C::real;
  const size_t n = (size_t)P.nx * P.ny, plane = (size_t)P.ny * P.pitch;
  const R inv = gscale_inv<typename C::gs, R>(P);
  double bad = 0, umax = 0, mx = 0, my = 0, mass = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % P.nx), y = (int)(i / P.nx);
    const size_t idx = (size_t)y * P.pitch + x;
    const double2 uv = u_value(u[idx]);
    bad += (isfinite(uv.x) ? 0.0 : 1.0) + (isfinite(uv.y) ? 0.0 : 1.0);
    umax = fmax(umax, fmax(fabs(uv.x), fabs(uv.y)));
    double r = 0, ax = 0, ay = 0;
    for (int q = 0; q < 9; ++q) {
      const double v = (double)(gload(g, q * plane + idx, inv) * inv);
      bad += isfinite(v) ? 0.0 : 1.0;
      r += v;
      ax += ex(q) * v;
      ay += ey(q) * v;
    }
    mass += r;
    mx += P.c * ax;
    my += P.c * ay;
  }
  __shared__ double sh[5][kMonThreads / 32];
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  bad = warp_sum(bad);
  umax = warp_max(umax);
  mx = warp_sum(mx);
  my = warp_sum(my);
  mass = warp_sum(mass);
  if (lane == 0) {
    sh[0][w] = bad;
    sh[1][w] = umax;
    sh[2][w] = mx;
    sh[3][w] = my;
    sh[4][w] = mass;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double o[5] = {0, 0, 0, 0, 0};
    for (int j = 0; j < kMonThreads / 32; ++j) {
      o[0] += sh[0][j];
      o[1] = fmax(o[1], sh[1][j]);
      o[2] += sh[2][j];
      o[3] += sh[3][j];
      o[4] += sh[4][j];
    }
    for (int m = 0; m < 5; ++m) partials[(size_t)blockIdx.x * 5 + m] = o[m];
  }
}

// final pass over nblocks partials; out[0..4] = bad, max|u|, momentum x, y, mass;
// out[5] = 1 if anything was non-finite (a sticky flag: never cleared here);
// out[6] = the iteration of the first monitor that set it
static __global__ void monitor_final_kernel(const double *partials, int nblocks, double *out, double k) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double o[5] = {0, 0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b) {
    o[0] += partials[(size_t)b * 5 + 0];
    o[1] = fmax(o[1], partials[(size_t)b * 5 + 1]);
    o[2] += partials[(size_t)b * 5 + 2];
    o[3] += partials[(size_t)b * 5 + 3];
    o[4] += partials[(size_t)b * 5 + 4];
  }
  for (int m = 0; m < 5; ++m) out[m] = o[m];
  if ((o[0] > 0 || !isfinite(o[1])) && out[5] == 0.0) {
    out[5] = 1.0;
    out[6] = k;
  }
}

// Grid error norms of Sect. 4 (Eq. griderror) against a reference field
// u_ref [ny][nx][2]: per-block partials of sum |u - u_ref|^2, max over nodes
// of max(|du_1|, |du_2|) and sum |u_ref|^2 (warp shuffle, then the block),
// then a fixed-order final pass: out = {E2, Einf, ||u_ref||_2} with
// E2 = ||du||_2 / (n ||u_ref||_2), Einf = ||du||_inf / ||u_ref||_2.
template <class C>
__global__ void __launch_bounds__(kMonThreads) grid_error_kernel(const Params P, const typename C::us *u,
                                                                 const double *uref, double *partials) {
  const size_t n = (size_t)P.nx * P.ny;
  double d2 = 0, dmax = 0, r2 = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % P.nx), y = (int)(i / P.nx);
    const double2 uv = u_value(u[(size_t)y * P.pitch + x]);
    const double rx = uref[2 * i], ry = uref[2 * i + 1];
    const double dx = uv.x - rx, dy = uv.y - ry;
    d2 += dx * dx + dy * dy;
    dmax = fmax(dmax, fmax(fabs(dx), fabs(dy)));
    r2 += rx * rx + ry * ry;
  }
  __shared__ double sh[3][kMonThreads / 32];
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  d2 = warp_sum(d2);
  dmax = warp_max(dmax);
  r2 = warp_sum(r2);
  if (lane == 0) {
    sh[0][w] = d2;
    sh[1][w] = dmax;
    sh[2][w] = r2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double o[3] = {0, 0, 0};
    for (int j = 0; j < kMonThreads / 32; ++j) {
      o[0] += sh[0][j];
      o[1] = fmax(o[1], sh[1][j]);
      o[2] += sh[2][j];
    }
    for (int m = 0; m < 3; ++m) partials[(size_t)blockIdx.x * 3 + m] = o[m];
  }
}

static __global__ void grid_error_final_kernel(const double *partials, int nblocks, double nodes, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double d2 = 0, dmax = 0, r2 = 0;
  for (int b = 0; b < nblocks; ++b) {
    d2 += partials[(size_t)b * 3 + 0];
    dmax = fmax(dmax, partials[(size_t)b * 3 + 1]);
    r2 += partials[(size_t)b * 3 + 2];
  }
  const double rn = sqrt(r2);
  out[0] = sqrt(d2) / (nodes * rn);
  out[1] = dmax / rn;
  out[2] = rn;
}

template <class C>
cudaError_t launch_grid_error(const Params &P, const void *u, const double *uref, double *partials, int nblocks,
                              double *out3, cudaStream_t st) {
  grid_error_kernel<C><<<nblocks, kMonThreads, 0, st>>>(P, (const typename C::us *)u, uref, partials);
  grid_error_final_kernel<<<1, 32, 0, st>>>(partials, nblocks, (double)P.nx * P.ny, out3);
  return cudaGetLastError();
}

template <class C>
__global__ void probe_kernel(const Params P, const typename C::us *u, const int32_t *idx, int n, double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int node = idx[i];
  const int x = node % P.nx, y = node / P.nx;
  const double2 uv = u_value(u[(size_t)y * P.pitch + x]);
  out[2 * i] = uv.x;
  out[2 * i + 1] = uv.y;
}

// ------------------------------------------------------------------ launchers
template <class C>
cudaError_t launch_init(const Params &P, void *g, void *u, void *b, const double *u0, const double *v0, cudaStream_t st) {
  dim3 grid((P.nx + C::TX - 1) / C::TX, (P.ny + C::TY - 1) / C::TY);
  init_kernel<C><<<grid, C::NT, 0, st>>>(P, (typename C::gs *)g, (typename C::us *)u, (typename C::real *)b, u0, v0);
  return cudaGetLastError();
}

template <class C>
cudaError_t launch_fields(const Params &P, const void *g, const void *u, double *uo, double *vo, double *Po,
                          cudaStream_t st) {
  dim3 grid((P.nx + C::TX - 1) / C::TX, (P.ny + C::TY - 1) / C::TY);
  fields_kernel<C><<<grid, C::NT, 0, st>>>(P, (const typename C::gs *)g, (const typename C::us *)u, uo, vo, Po);
  return cudaGetLastError();
}

template <class C>
cudaError_t launch_monitor(const Params &P, const void *g, const void *u, double *partials, int nblocks, double *out6,
                           int64_t k, cudaStream_t st) {
  monitor_kernel<C><<<nblocks, kMonThreads, 0, st>>>(P, (const typename C::gs *)g, (const typename C::us *)u, partials);
  monitor_final_kernel<<<1, 32, 0, st>>>(partials, nblocks, out6, (double)k);
  return cudaGetLastError();
}

template <class C>
cudaError_t launch_probe(const Params &P, const void *u, const int32_t *idx, int n, double *out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  probe_kernel<C><<<(n + 127) / 128, 128, 0, st>>>(P, (const typename C::us *)u, idx, n, out);
  return cudaGetLastError();
}

}  // namespace lbs
