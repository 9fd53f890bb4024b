// Exact Riemann solver for the ideal gas, device side (Sec. 3.3: exact
// solver with a treatment of vacuum; the mathematics is that of the 1D Euler
// Riemann problem).
//
// The star pressure p* is the root of
//   f(p) = f_L(p) + f_R(p) + (u_R - u_L),
//   f_K(p) = (p - p_K) sqrt(A_K / (p + B_K))                      p > p_K (shock)
//          = 2 c_K / (gamma-1) ((p/p_K)^z - 1),  z=(gamma-1)/(2gamma)  p <= p_K (rarefaction)
//   A_K = 2 / ((gamma+1) rho_K), B_K = (gamma-1)/(gamma+1) p_K,
// found by Newton's method to the relative change 2|dp|/(p_new+p_old) < tol
// from a starting value, then sampled at x/t = 0.  The rarefaction derivative
// uses (p/p_K)^(z-1) = (p/p_K)^z / (p/p_K) so one power serves f and f'.
// Vacuum generated between two rarefactions (2(c_L+c_R)/(gamma-1) <= u_R-u_L)
// is handled in closed form; the extrapolated states reaching this solver are
// always positive (non-positive ones fall back to first order before).
//
// FP32 form: the iteration runs in float.  Near vacuum and in strong
// rarefactions float cannot resolve the relative tolerance (f is a
// difference of terms ~2c/(gamma-1) that cancel), so once an iterate falls
// below GUARD * min(p_L, p_R), or the float loop has not converged after
// FLOAT_ITERS iterations, the solve continues in FP64 (pressure functions,
// step and convergence test), and the face is counted.
#pragma once

#include <cuda_runtime.h>
#include <float.h>

#include "amm_internal.cuh"

namespace amm {


__device__ __forceinline__ double xpow(double a, double b) { return pow(a, b); }
__device__ __forceinline__ float xpow(float a, float b) { return __powf(a, b); }
__device__ __forceinline__ double xsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float xsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double xrsqrt(double a) { return rsqrt(a); }
__device__ __forceinline__ float xrsqrt(float a) { return rsqrtf(a); }

// Explicitly rounded products, sums and fused multiply-adds: the compiler
// neither fuses nor splits them, so a formula written with them rounds the
// same in every kernel it is inlined into.  Whether a plain a * b + c is
// fused depends on where the compiler places the product relative to the
// branches of an inlined FP64 division or square root, which differs
// between kernels.  The per-phase kernels and the persistent step kernel
// must agree bit for bit.
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// a . b of two 3-vectors, x first
template <typename real>
__device__ __forceinline__ real rn_dot3(real ax, real ay, real az, real bx, real by, real bz) {
  return rn_fma(az, bz, rn_fma(ay, by, rn_mul(ax, bx)));
}

// f_K(p) and f_K'(p)
template <typename real>
__device__ __forceinline__ void wave_curve(real p, real rhoK, real pK, real cK, const GasC<real>& G, real& f,
                                           real& df) {
  if constexpr (sizeof(real) == 4) {
    // FP32: both branches, selected.  The sides of a warp's faces split
    // between shocks and rarefactions, so a branch would run both anyway;
    // unconditional, the per-side constants leave the Newton loop.
    const real A = G.two_gp1 / rhoK;
    const real id = (real)1 / (p + G.gm1_gp1 * pK);
    const real q = xsqrt(A * id);
    const real fs = (p - pK) * q;
    const real dfs = q * ((real)1 - (real)0.5 * (p - pK) * id);
    const real pr = p / pK;
    const real prz = xpow(pr, G.z);
    const real fr = G.two_gm1 * cK * (prz - (real)1);
    const real dfr = prz / (pr * rhoK * cK);
    const bool shock = p > pK;
    f = shock ? fs : fr;
    df = shock ? dfs : dfr;
  } else if (p > pK) {
    const real A = G.two_gp1 / rhoK;
    const real B = G.gm1_gp1 * pK;
    const real q = xsqrt(A / (p + B));
    f = (p - pK) * q;
    df = q * ((real)1 - (real)0.5 * (p - pK) / (p + B));
  } else {
    const real pr = p / pK;
    const real prz = xpow(pr, G.z);
    f = G.two_gm1 * cK * (prz - (real)1);
    df = prz / (pr * rhoK * cK);
  }
}

// Linearised (primitive-variable) star pressure, clipped at 0, and the
// two-shock estimate evaluated at it.
template <typename real>
__device__ __forceinline__ real linearised_pstar(real rhoL, real uL, real pL, real cL, real rhoR, real uR, real pR,
                                                 real cR) {
  const real ppv = (real)0.5 * (pL + pR) - (real)0.125 * (uR - uL) * (rhoL + rhoR) * (cL + cR);
  return ppv > (real)0 ? ppv : (real)0;
}

template <typename real>
__device__ __forceinline__ real two_shock_pstar(real rhoL, real uL, real pL, real rhoR, real uR, real pR, real ppv,
                                                const GasC<real>& G) {
  const real gL = xsqrt((G.two_gp1 / rhoL) / (ppv + G.gm1_gp1 * pL));
  const real gR = xsqrt((G.two_gp1 / rhoR) / (ppv + G.gm1_gp1 * pR));
  return (gL * pL + gR * pR - (uR - uL)) / (gL + gR);
}

// Standard starting value: the linearised (primitive-variable) estimate when
// the pressure ratio is small and it lies between p_L and p_R, else the
// two-rarefaction estimate when it lies below both, else the two-shock
// estimate evaluated at the linearised pressure; floored positive.  With a
// proposal (`have`), the proposal replaces the two-shock estimate -- the one
// approximate branch: the two-rarefaction estimate is the exact star pressure
// when both waves are rarefactions, and the linearised one is kept where it
// passes its own test.
template <typename real>
__device__ __forceinline__ real standard_guess_ppv(real rhoL, real uL, real pL, real cL, real rhoR, real uR, real pR,
                                                   real cR, real ppv, const GasC<real>& G, bool have = false,
                                                   real proposal = (real)0) {
  const real du = uR - uL;
  const real pmin = pL < pR ? pL : pR, pmax = pL > pR ? pL : pR;
  real p0;
  if constexpr (sizeof(real) == 4) {
    // FP32: every estimate, selected (a warp's faces take all three, so
    // branches would run them all anyway)
    const bool pv = pmax <= (real)2 * pmin && ppv >= pmin && ppv <= pmax;
    const real num = cL + cR - (real)0.5 * G.gm1 * du;
    const real den = cL / xpow(pL, G.z) + cR / xpow(pR, G.z);
    const real ptr = xpow(num / den, G.inv_z);
    const real pts = have ? proposal : two_shock_pstar(rhoL, uL, pL, rhoR, uR, pR, ppv, G);
    p0 = pv ? ppv : (ppv < pmin ? ptr : pts);
  } else if (pmax / pmin <= (real)2 && ppv >= pmin && ppv <= pmax) {
    p0 = ppv;
  } else if (ppv < pmin) {
    const real num = cL + cR - (real)0.5 * G.gm1 * du;
    const real den = cL / xpow(pL, G.z) + cR / xpow(pR, G.z);
    p0 = xpow(num / den, G.inv_z);
  } else if (have) {
    p0 = proposal;
  } else {
    p0 = two_shock_pstar(rhoL, uL, pL, rhoR, uR, pR, ppv, G);
  }
  const real pfloor = (real)1e-10 * (real)0.5 * (pL + pR);
  return (p0 > pfloor) ? p0 : pfloor;
}

template <typename real>
__device__ __forceinline__ real standard_guess(real rhoL, real uL, real pL, real cL, real rhoR, real uR, real pR,
                                               real cR, const GasC<real>& G, bool have = false,
                                               real proposal = (real)0) {
  return standard_guess_ppv(rhoL, uL, pL, cL, rhoR, uR, pR, cR, linearised_pstar(rhoL, uL, pL, cL, rhoR, uR, pR, cR),
                            G, have, proposal);
}

struct RiemannInfo {
  int iters;
  int guard;      // finished in FP64
  int vacuum;
  int fail;       // hit the iteration cap
};

// State of the last Newton step: f_L, f_R and their derivatives at the
// previous iterate p_prev; u* at the final p follows to first order,
// u* = (u_L+u_R)/2 + (f_R - f_L + (f_R' - f_L')(p - p_prev))/2, with an error
// of order (p - p_prev)^2, far below the tolerance.
template <typename real>
struct NewtonTail {
  real fL, dL, fR, dR, dp;
};

// The FP64 Newton loops also stop when f(p) vanishes to rounding (|f| within
// RESIDUAL_ULPS ulps of the size of its terms): p is then the root in working
// precision.  Near vacuum f is a small difference of large terms and the
// relative change of p cannot fall below a 1e-12 tolerance.
constexpr double RESIDUAL_ULPS = 64.0;

// Newton iteration for p*; returns p* in `real`, with the FP64 guard in the
// FP32 form.  iterations counted in info.
template <typename real>
__device__ __forceinline__ real newton_pstar(real p, real rhoL, real uL, real pL, real cL, real rhoR, real uR,
                                             real pR, real cR, const GasC<real>& G, double tol, real tol_r, int maxit,
                                             RiemannInfo& info, NewtonTail<real>& tail) {
  const real du = uR - uL;
  int it = 0;
  bool conv = false;
  if constexpr (sizeof(real) == 8) {
    while (it < maxit) {
      real fL, dL, fR, dR;
      wave_curve(p, rhoL, pL, cL, G, fL, dL);
      wave_curve(p, rhoR, pR, cR, G, fR, dR);
      const real f = fL + fR + du;
      if (fabs(f) <= RESIDUAL_ULPS * DBL_EPSILON * (fabs(fL) + fabs(fR) + fabs(du))) {
        tail.fL = fL; tail.dL = dL; tail.fR = fR; tail.dR = dR; tail.dp = (real)0;
        conv = true;
        break;
      }
      real pn = p - f / (dL + dR);
      if (!(pn > (real)0)) pn = (real)1e-3 * p;
      it++;
      const real ch = (real)2 * fabs(pn - p) / (pn + p);
      tail.fL = fL; tail.dL = dL; tail.fR = fR; tail.dR = dR; tail.dp = pn - p;
      p = pn;
      if (ch < (real)tol) {
        conv = true;
        break;
      }
    }
  } else {
    constexpr int FLOAT_ITERS = 12;
    const float tol_f = (float)tol_r;   // the tolerance in FP32, converted once on the host
    const float guard_p = 1e-3f * (pL < pR ? (float)pL : (float)pR);
    bool to64 = false;
    while (it < maxit) {
      if (it >= FLOAT_ITERS || (float)p < guard_p) {
        to64 = true;
        break;
      }
      real fL, dL, fR, dR;
      wave_curve(p, rhoL, pL, cL, G, fL, dL);
      wave_curve(p, rhoR, pR, cR, G, fR, dR);
      real pn = p - (fL + fR + du) / (dL + dR);
      if (!(pn > (real)0)) pn = (real)1e-3 * p;
      it++;
      // 2 |dp| / (p_new + p_old) < tol, without the division
      const bool done = (real)2 * fabsf((float)(pn - p)) < tol_f * (pn + p);
      tail.fL = fL; tail.dL = dL; tail.fR = fR; tail.dR = dR; tail.dp = pn - p;
      p = pn;
      if (done) {
        conv = true;
        break;
      }
    }
    if (to64) {
      info.guard = 1;
      const GasC<double> G64((double)G.g);
      double pd = (double)p;
      const double rL = rhoL, uLd = uL, pLd = pL, rR = rhoR, uRd = uR, pRd = pR;
      const double cLd = sqrt(G64.g * pLd / rL), cRd = sqrt(G64.g * pRd / rR);
      const double dud = uRd - uLd;
      while (it < maxit) {
        double fL, dL, fR, dR;
        wave_curve(pd, rL, pLd, cLd, G64, fL, dL);
        wave_curve(pd, rR, pRd, cRd, G64, fR, dR);
        const double f = fL + fR + dud;
        if (fabs(f) <= RESIDUAL_ULPS * DBL_EPSILON * (fabs(fL) + fabs(fR) + fabs(dud))) {
          tail.fL = (real)fL; tail.dL = (real)dL; tail.fR = (real)fR; tail.dR = (real)dR; tail.dp = (real)0;
          conv = true;
          break;
        }
        double pn = pd - f / (dL + dR);
        if (!(pn > 0.0)) pn = 1e-3 * pd;
        it++;
        const double ch = 2.0 * fabs(pn - pd) / (pn + pd);
        tail.fL = (real)fL; tail.dL = (real)dL; tail.fR = (real)fR; tail.dR = (real)dR; tail.dp = (real)(pn - pd);
        pd = pn;
        if (ch < tol) {
          conv = true;
          break;
        }
      }
      p = (real)pd;
    }
  }
  info.iters = it;
  info.fail = conv ? 0 : 1;
  return p;
}

// Sampled state at x/t = 0 of the Riemann problem (rho, u, p per side).
// Returns side of the contact (0: left, 1: right) for the transverse
// velocity; rho = P = 0 inside generated vacuum.  pstar: the star pressure
// (0 when vacuum is generated).
// cL, cR: the sides' sound speeds; ppv: the linearised star pressure (the
// caller may have formed them already, for the proposal's gate).
template <typename real>
__device__ __forceinline__ int riemann_sample_c(real rhoL, real uL, real pL, real rhoR, real uR, real pR, real cL,
                                                real cR, real ppv, const GasC<real>& G, double tol, real tol_r,
                                                int maxit, bool have_guess, real guess, real& rhoF, real& uF, real& pF,
                                                RiemannInfo& info, real& pstar) {
  pstar = (real)0;
  info.iters = 0;
  info.guard = 0;
  info.vacuum = 0;
  info.fail = 0;
  if (G.two_gm1 * (cL + cR) <= uR - uL) {
    // two rarefactions with vacuum between them
    info.vacuum = 1;
    const real frontL = uL + G.two_gm1 * cL;
    const real frontR = uR - G.two_gm1 * cR;
    if ((real)0 <= frontL) {
      if ((real)0 <= uL - cL) {
        rhoF = rhoL; uF = uL; pF = pL;
      } else {
        const real c = G.two_gp1 * cL + G.gm1_gp1 * uL;
        const real r = c / cL;
        uF = c;
        rhoF = rhoL * xpow(r, G.fan_rho);
        pF = pL * xpow(r, G.fan_p);
      }
      return 0;
    }
    if ((real)0 >= frontR) {
      if ((real)0 >= uR + cR) {
        rhoF = rhoR; uF = uR; pF = pR;
      } else {
        const real c = G.two_gp1 * cR - G.gm1_gp1 * uR;
        const real r = c / cR;
        uF = -c;
        rhoF = rhoR * xpow(r, G.fan_rho);
        pF = pR * xpow(r, G.fan_p);
      }
      return 1;
    }
    rhoF = (real)0; uF = (real)0.5 * (frontL + frontR); pF = (real)0;
    return 0;
  }
  const real p0 = standard_guess_ppv(rhoL, uL, pL, cL, rhoR, uR, pR, cR, ppv, G, have_guess, guess);
  NewtonTail<real> nt;
  const real ps = newton_pstar(p0, rhoL, uL, pL, cL, rhoR, uR, pR, cR, G, tol, tol_r, maxit, info, nt);
  pstar = ps;
  const real us = (real)0.5 * (uL + uR) + (real)0.5 * ((nt.fR - nt.fL) + (nt.dR - nt.dL) * nt.dp);
  // the side the face sees (the contact's upwind side): s = +1 left, -1
  // right; the right side's formulas are the left side's with the velocity
  // signs flipped (products with s are exact), so one path serves both
  const int side = ((real)0 <= us) ? 0 : 1;
  const real s = side ? (real)-1 : (real)1;
  const real rhoK = side ? rhoR : rhoL, uK = side ? uR : uL, pK = side ? pR : pL, cK = side ? cR : cL;
  const real r = ps / pK;
  if constexpr (sizeof(real) == 4) {
    // FP32: the shock and rarefaction cases evaluated and selected; only the
    // sonic rarefaction (the face inside the fan, rare) branches
    const bool shock = ps > pK;
    const real sq = xsqrt(G.shock_a * r + G.shock_b);
    const real lr = __log2f(r);
    const real rz = exp2f(G.z * lr), rig = exp2f(G.inv_g * lr);
    const bool orig = shock ? ((real)0 <= s * (uK - s * cK * sq)) : ((real)0 <= s * (uK - s * cK));
    const bool fan = !shock && !orig && !((real)0 > s * (us - s * cK * rz));
    const real rho_star = shock ? rhoK * (r + G.gm1_gp1) / (G.gm1_gp1 * r + (real)1) : rhoK * rig;
    rhoF = orig ? rhoK : rho_star;
    uF = orig ? uK : us;
    pF = orig ? pK : ps;
    if (fan) {
      const real c = G.two_gp1 * cK + s * G.gm1_gp1 * uK;
      const real q = c / cK;
      uF = s * c;
      rhoF = rhoK * xpow(q, G.fan_rho);
      pF = pK * xpow(q, G.fan_p);
    }
  } else if (ps > pK) {
    const real SK = uK - s * cK * xsqrt(G.shock_a * r + G.shock_b);
    if ((real)0 <= s * SK) {
      rhoF = rhoK; uF = uK; pF = pK;
    } else {
      rhoF = rhoK * (r + G.gm1_gp1) / (G.gm1_gp1 * r + (real)1); uF = us; pF = ps;
    }
  } else {
    if ((real)0 <= s * (uK - s * cK)) {
      rhoF = rhoK; uF = uK; pF = pK;
    } else {
      const real tail = us - s * cK * xpow(r, G.z);
      if ((real)0 > s * tail) {
        rhoF = rhoK * xpow(r, G.inv_g); uF = us; pF = ps;
      } else {
        const real c = G.two_gp1 * cK + s * G.gm1_gp1 * uK;
        const real q = c / cK;
        uF = s * c;
        rhoF = rhoK * xpow(q, G.fan_rho);
        pF = pK * xpow(q, G.fan_p);
      }
    }
  }
  return side;
}

template <typename real>
__device__ __forceinline__ int riemann_sample(real rhoL, real uL, real pL, real rhoR, real uR, real pR,
                                              const GasC<real>& G, double tol, real tol_r, int maxit, bool have_guess,
                                              real guess, real& rhoF, real& uF, real& pF, RiemannInfo& info,
                                              real& pstar) {
  const real cL = xsqrt(G.g * pL / rhoL), cR = xsqrt(G.g * pR / rhoR);
  return riemann_sample_c(rhoL, uL, pL, rhoR, uR, pR, cL, cR, linearised_pstar(rhoL, uL, pL, cL, rhoR, uR, pR, cR), G,
                          tol, tol_r, maxit, have_guess, guess, rhoF, uF, pF, info, pstar);
}

}  // namespace amm
