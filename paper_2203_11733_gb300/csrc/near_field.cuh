// FP64 closed forms of the Galerkin double integrals over pairs of
// axis-aligned rectangles, as 16-term corner sums of antiderivatives.
//
// Single layer (Sec. 3.4): int int 1/|x - y|.  Parallel panels: F(u,v,w)
// with d^4F/du^2dv^2 = 1/rho; perpendicular panels: H(u,v,w) with
// d^4H/du^2dvdw = 1/rho (rho = sqrt(u^2 + v^2 + w^2)).
//
// Double layer (Sec. 4, the integrals Q_ij of the multi-dielectric system):
// int int <x - y, n_j> / |x - y|^3 for the normal n_j = +e_k of panel j.
// For parallel panels <x - y, n_j> = w, the plane offset, and the integrand
// w / rho^3 is the mixed derivative d^2/du dv of atan(u v / (w rho)); its
// second antiderivative in u and in v is
//     Phi(u,v,w) = u v atan(u v / (w rho)) + u w ln(u + rho) + v w ln(v + rho)
//                  - (u w / 2) ln(v^2 + w^2) - (v w / 2) ln(u^2 + w^2) - w rho.
// For perpendicular panels <x - y, n_j> = v, the coordinate of x along j's
// normal measured from j's plane, and v / rho^3 = -d/dv (1/rho); the
// antiderivative with the derivative pattern of H (second in u, first in v
// and w) is
//     Theta(u,v,w) = u v atan(u w / (v rho)) - u w ln(u + rho)
//                    - ((u^2 - v^2) / 2) ln(w + rho) + w rho / 2
// (terms that cancel in the corner sum dropped).  Both were checked by
// differentiating them back to their kernels.
#pragma once

namespace {

// 1/sqrt(x) in FP64: single-precision estimate refined by one Newton step
// y <- y + y (1 - x y^2) / 2 (relative error about 1.5 e0^2 < 1e-13).
__device__ __forceinline__ double rsq64(double x)
{
    double y = (double)rsqrtf((float)x);
    double e = fma(-x * y, y, 1.0);
    return fma(0.5 * y, e, y);
}

// coef * ln(t + rho) with rho = sqrt(t^2 + r2); 0 * ln 0 -> 0; the t < 0 branch
// uses ln(t + rho) = ln(r2 / (rho - t)) to avoid cancellation.
__device__ __forceinline__ double xlog(double coef, double t, double r2, double rho)
{
    if (coef == 0.0) return 0.0;
    return (t >= 0.0) ? coef * log(t + rho) : coef * log(r2 / (rho - t));
}

// F(u,v,w) = v/2 (u^2-w^2) ln(v+rho) + u/2 (v^2-w^2) ln(u+rho)
//            - (u^2+v^2-2w^2) rho/6 - u v w atan(u v/(w rho))
__device__ __noinline__ double F_par(double u, double v, double w)
{
    double u2 = u * u, v2 = v * v, w2 = w * w;
    double rho = sqrt(u2 + v2 + w2);
    double r = xlog(0.5 * v * (u2 - w2), v, u2 + w2, rho) + xlog(0.5 * u * (v2 - w2), u, v2 + w2, rho) -
               (u2 + v2 - 2.0 * w2) * rho * (1.0 / 6.0);
    double uvw = u * v * w;
    if (uvw != 0.0) r -= uvw * atan(u * v / (w * rho));
    return r;
}

// H(u,v,w) = u v w ln(u+rho) + w(3u^2-w^2)/6 ln(v+rho) + v(3u^2-v^2)/6 ln(w+rho)
//            - v w rho/3 - u w^2/2 atan(uv/(w rho)) - u v^2/2 atan(uw/(v rho))
//            - u^3/6 atan(vw/(u rho))
__device__ __noinline__ double H_orth(double u, double v, double w)
{
    double u2 = u * u, v2 = v * v, w2 = w * w;
    double rho = sqrt(u2 + v2 + w2);
    double r = xlog(u * v * w, u, v2 + w2, rho) +
               xlog(w * (3.0 * u2 - w2) * (1.0 / 6.0), v, u2 + w2, rho) +
               xlog(v * (3.0 * u2 - v2) * (1.0 / 6.0), w, u2 + v2, rho) - v * w * rho * (1.0 / 3.0);
    if (u * w != 0.0 && v != 0.0) r -= 0.5 * u * w2 * atan(u * v / (w * rho));
    if (u * v != 0.0 && w != 0.0) r -= 0.5 * u * v2 * atan(u * w / (v * rho));
    if (u != 0.0 && v * w != 0.0) r -= (u * u2 * (1.0 / 6.0)) * atan(v * w / (u * rho));
    return r;
}

// F and Phi at one corner together (parallel panels, w != 0): they share
// rho, ln(u + rho), ln(v + rho) and atan(u v / (w rho)).
__device__ __noinline__ void FPhi_par(double u, double v, double w, double& f, double& phi)
{
    double u2 = u * u, v2 = v * v, w2 = w * w;
    double rho = sqrt(u2 + v2 + w2);
    const double lu = (u != 0.0) ? xlog(1.0, u, v2 + w2, rho) : 0.0;   // ln(u + rho)
    const double lv = (v != 0.0) ? xlog(1.0, v, u2 + w2, rho) : 0.0;   // ln(v + rho)
    const double at = (u * v != 0.0) ? atan(u * v / (w * rho)) : 0.0;
    f = 0.5 * v * (u2 - w2) * lv + 0.5 * u * (v2 - w2) * lu - (u2 + v2 - 2.0 * w2) * rho * (1.0 / 6.0) -
        u * v * w * at;
    phi = u * w * lu + v * w * lv - 0.5 * u * w * log(v2 + w2) - 0.5 * v * w * log(u2 + w2) - w * rho + u * v * at;
}

// H and Theta at one corner together (perpendicular panels): they share rho,
// ln(u + rho), ln(w + rho) and atan(u w / (v rho)).
__device__ __noinline__ void HTheta_orth(double u, double v, double w, double& h, double& theta)
{
    double u2 = u * u, v2 = v * v, w2 = w * w;
    double rho = sqrt(u2 + v2 + w2);
    // ln(u + rho) and ln(w + rho), 0 where the argument vanishes (their
    // coefficients vanish there too: the 0 ln 0 limits)
    const double lu = (v2 + w2 != 0.0 || u > 0.0) ? xlog(1.0, u, v2 + w2, rho) : 0.0;
    const double lw = (u2 + v2 != 0.0 || w > 0.0) ? xlog(1.0, w, u2 + v2, rho) : 0.0;
    const double a_uw = (u * v != 0.0 && w != 0.0) ? atan(u * w / (v * rho)) : 0.0;
    h = u * v * w * lu + xlog(w * (3.0 * u2 - w2) * (1.0 / 6.0), v, u2 + w2, rho) +
        v * (3.0 * u2 - v2) * (1.0 / 6.0) * lw - v * w * rho * (1.0 / 3.0) - 0.5 * u * v2 * a_uw;
    if (u * w != 0.0 && v != 0.0) h -= 0.5 * u * w2 * atan(u * v / (w * rho));
    if (u != 0.0 && v * w != 0.0) h -= (u * u2 * (1.0 / 6.0)) * atan(v * w / (u * rho));
    theta = -u * w * lu - 0.5 * (u2 - v2) * lw + 0.5 * w * rho + u * v * a_uw;
}

}  // namespace
