// PLIC geometry in FP64 (Section 2: the interface in a cell is a plane).
//
// Volume of the unit cube below the plane m.xi = d, and its inverse. After
// reflecting negative components and normalising so the sorted components
// b1 <= b2 <= b3 sum to one, the half-range a in [0, 1/2] splits into five
// polynomial pieces (inclusion-exclusion of the corner simplex, a^3 minus
// the simplices cut off beyond each vertex). Each piece is written here in
// factored form, e.g. a^3 - (a-b1)^3 = b1 (a^2 + a p + p^2) with p = a - b1,
// so that dividing by a small b1 never amplifies cancellation: the
// subtracted remainders (q^3/b1 with q < b1, and so on) are bounded by the
// leading terms. The upper half follows from V(a) = 1 - V(1 - a).
#pragma once

#include <cuda_runtime.h>

namespace plic {

__device__ __forceinline__ void sort3(double& x, double& y, double& z) {
    double t;
    if (x > y) { t = x; x = y; y = t; }
    if (y > z) { t = y; y = z; z = t; }
    if (x > y) { t = x; x = y; y = t; }
}

// piece C: b2 <= a < min(b1+b2, b3)  (requires b1 > 0)
__device__ __forceinline__ double vol_C(double b1, double b2, double b3, double a) {
    const double p = a - b1, q = a - b2;
    return (a * a + a * p + p * p - q * q * q / b1) / (6.0 * b2 * b3);
}
// piece E: max(b3) <= a <= 1/2 with b1+b2 >= b3
__device__ __forceinline__ double vol_E(double b1, double b2, double b3, double a) {
    const double p = a - b1, s = a - b2, r = a - b3;
    const double t = b1 > 0.0 ? (s * s * s + r * r * r) / b1 : 0.0;
    return (a * a + a * p + p * p - t) / (6.0 * b2 * b3);
}

// V(a) for sorted, normalised b and a in [0, 1/2]
__device__ __forceinline__ double vol_half(double b1, double b2, double b3, double a) {
    if (a <= 0.0) return 0.0;
    if (a < b1) return a * a * a / (6.0 * b1 * b2 * b3);
    if (a < b2) return (3.0 * a * (a - b1) + b1 * b1) / (6.0 * b2 * b3);
    const double b12 = b1 + b2;
    if (a < fmin(b12, b3)) return vol_C(b1, b2, b3, a);
    if (a < b3) return (2.0 * a - b12) / (2.0 * b3);
    return vol_E(b1, b2, b3, a);
}

// Liquid volume fraction of the unit cube below m.xi = d (any signs of m).
__device__ __forceinline__ double volume(double m0, double m1, double m2, double d) {
    if (m0 < 0.0) { d -= m0; m0 = -m0; }
    if (m1 < 0.0) { d -= m1; m1 = -m1; }
    if (m2 < 0.0) { d -= m2; m2 = -m2; }
    const double S = m0 + m1 + m2;
    if (!(S > 0.0)) return d >= 0.0 ? 1.0 : 0.0;
    const double a = d / S;
    if (a <= 0.0) return 0.0;
    if (a >= 1.0) return 1.0;
    double b1 = m0 / S, b2 = m1 / S, b3 = m2 / S;
    sort3(b1, b2, b3);
    b3 = 1.0 - b1 - b2;
    return a <= 0.5 ? vol_half(b1, b2, b3, a) : 1.0 - vol_half(b1, b2, b3, 1.0 - a);
}

__device__ __forceinline__ double rcp_approx64(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    return r;
}

// Normalised plane constant a in [0, 1/2] with vol_half(b, a) = V, written
// for warps whose lanes fall in different pieces: the divisions are hoisted
// (reciprocals formed once), and the two cubic pieces C and E share one
// Newton loop (E adds the term of the third vertex), so lanes in C and E
// run the same instructions. Newton steps use an approximate reciprocal of
// the derivative; the safeguarding bracket keeps every iterate inside the
// piece, and the iteration stops on a relative step or bracket of 2.3e-16.
__device__ __forceinline__ double solve_half(double b1, double b2, double b3, double V) {
    if (V <= 0.0) return 0.0;
    if (b2 <= 0.0) return V;  // axis-aligned plane: V(a) = a
    const double i6 = 1.0 / (6.0 * b2 * b3);  // 1 / (6 b2 b3)
    const double ib1 = b1 > 0.0 ? 1.0 / b1 : 0.0;
    const double V1 = b1 * b1 * i6;
    if (V < V1) return cbrt(6.0 * b1 * b2 * b3 * V);
    const double V2 = (3.0 * b2 * (b2 - b1) + b1 * b1) * i6;
    if (V < V2) return 0.5 * b1 + sqrt(fmax(2.0 * b2 * b3 * V - b1 * b1 / 12.0, 0.0));
    const double b12 = b1 + b2;
    double lo, hi, Vlo, Vhi;
    bool e_piece;
    if (b12 <= b3) {
        const double V3 = b12 / (2.0 * b3);
        if (!(V < V3 && b1 > 0.0)) return V * b3 + 0.5 * b12;  // piece D
        lo = b2; hi = b12; Vlo = V2; Vhi = V3; e_piece = false;
    } else {
        double V3 = V2;
        if (b1 > 0.0) {
            const double p = b3 - b1, q = b3 - b2;
            V3 = (b3 * b3 + b3 * p + p * p - q * q * q * ib1) * i6;
        }
        if (V < V3) { lo = b2; hi = b3; Vlo = V2; Vhi = V3; e_piece = false; }
        else { lo = b3; hi = 0.5; Vlo = V3; Vhi = 0.5; e_piece = true; }
    }
    const double i2 = 3.0 * i6;  // 1 / (2 b2 b3)
    double a = (Vhi > Vlo) ? lo + (hi - lo) * (V - Vlo) / (Vhi - Vlo) : 0.5 * (lo + hi);
    for (int it = 0; it < 48; ++it) {
        const double p = a - b1, q = a - b2, r = e_piece ? a - b3 : 0.0;
        const double f = (a * a + a * p + p * p - (q * q * q + r * r * r) * ib1) * i6 - V;
        const double df = (a + p - (q * q + r * r) * ib1) * i2;
        if (f == 0.0) break;
        if (f > 0.0) hi = a; else lo = a;
        const double dn = df > 0.0 ? f * rcp_approx64(df) : 0.0;
        // a Newton correction below the rounding of a means a is the root to
        // working precision; take it before the bracket test, which would
        // reject the unchanged a (it sits on the bracket) and bisect
        if (df > 0.0 && fabs(dn) <= 2.3e-16 * a) {
            a -= dn;
            break;
        }
        double an = df > 0.0 ? a - dn : 0.5 * (lo + hi);
        if (!(an > lo && an < hi)) an = 0.5 * (lo + hi);
        const double step = fabs(an - a);
        a = an;
        if (step <= 2.3e-16 * a || hi - lo <= 2.3e-16 * hi) break;
    }
    return a;
}

// Plane constant d with volume(m, d) = alpha, 0 < alpha < 1, m != 0.
__device__ __forceinline__ double plane_constant(double m0, double m1, double m2, double alpha) {
    double off = 0.0;
    if (m0 < 0.0) { off += m0; m0 = -m0; }
    if (m1 < 0.0) { off += m1; m1 = -m1; }
    if (m2 < 0.0) { off += m2; m2 = -m2; }
    const double S = m0 + m1 + m2;
    if (!(S > 0.0)) return 0.0;
    const double iS = 1.0 / S;
    double b1 = m0 * iS, b2 = m1 * iS, b3 = m2 * iS;
    sort3(b1, b2, b3);
    b3 = 1.0 - b1 - b2;
    const double V = alpha <= 0.5 ? alpha : 1.0 - alpha;
    double a = solve_half(b1, b2, b3, V);
    if (alpha > 0.5) a = 1.0 - a;
    return a * S + off;
}

// Which branch of plane_constant a cell takes, estimated in FP32 (0: a
// closed form with no piece search, 1: cube-corner piece (cube root), 2:
// the quadratic piece (square root), 3: the linear piece, 4 and 5: the two
// cubic pieces (Newton)). The estimate only orders the cells so that the
// lanes of a warp take the same branch; plane_constant decides each cell's
// branch itself, so a wrong estimate near a piece boundary changes nothing.
__device__ __forceinline__ int plane_piece_estimate(double n0, double n1, double n2, double alpha) {
    float m0 = fabsf((float)n0), m1 = fabsf((float)n1), m2 = fabsf((float)n2);
    const float S = m0 + m1 + m2;
    if (!(S > 0.f)) return 0;
    const float iS = 1.f / S;
    float b1 = m0 * iS, b2 = m1 * iS, b3 = m2 * iS, t;
    if (b1 > b2) { t = b1; b1 = b2; b2 = t; }
    if (b2 > b3) { t = b2; b2 = b3; b3 = t; }
    if (b1 > b2) { t = b1; b1 = b2; b2 = t; }
    b3 = 1.f - b1 - b2;
    const float a = (float)alpha, V = a <= 0.5f ? a : 1.f - a;
    if (V <= 0.f || b2 <= 0.f) return 0;
    const float i6 = 1.f / (6.f * b2 * b3);
    if (V < b1 * b1 * i6) return 1;
    if (V < (3.f * b2 * (b2 - b1) + b1 * b1) * i6) return 2;
    const float b12 = b1 + b2;
    if (b12 <= b3) return (V < b12 / (2.f * b3) && b1 > 0.f) ? 4 : 3;
    float V3 = (3.f * b2 * (b2 - b1) + b1 * b1) * i6;
    if (b1 > 0.f) {
        const float p = b3 - b1, q = b3 - b2;
        V3 = (b3 * b3 + b3 * p + p * p - q * q * q / b1) * i6;
    }
    return V < V3 ? 4 : 5;
}

// Liquid fraction (of the whole cell) inside the donor slab of relative
// width c next to the face: the plus face when plus_side, else the minus
// face. The slab is rescaled to a unit cube along dir.
__device__ __forceinline__ double slab_fraction(double n0, double n1, double n2, double d, int dir,
                                                double c, bool plus_side) {
    double m[3] = {n0, n1, n2};
    if (plus_side) d -= m[dir] * (1.0 - c);
    m[dir] *= c;
    return c * volume(m[0], m[1], m[2], d);
}

}  // namespace plic
