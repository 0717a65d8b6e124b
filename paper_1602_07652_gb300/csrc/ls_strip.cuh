// ls_strip.cuh -- entries of the local matrices C^l of the layered decomposition.
//
// Sec. 3.1: layer l owns rows [l t, (l+1) t) of its direction's grid (t = n / L)
// and is extended by E rows on each side; local row r <-> row z = l t - E + r,
// r in [0, q), q = t + 2E.  Rows outside Omega are decoupled identity rows, so
// every strip has the same q.
// Sec. 3.3: C^l uses D^l = diag(xi^l m) plus a complex shift in the cut-off
// region; its outermost rows inside Omega use the boundary stencils of Omega.
// Readings (the paper's display of xi^l is empty): xi^l = 1 on the layer and on
// its two halo rows (compatibility with C), then the cubic S(tau) = 1 - 3 tau^2
// + 2 tau^3, tau = (dist - 1) / (E - 1), over the remaining E - 1 rows, reaching 0
// on the outermost row; the shifted contrast is m^l = xi^l m + i (c/w)(1 - xi^l).
// Then C^l(k, k+d) = alpha^{t(k)}_d + w^2 beta^{t(k)}_d m^l_{k+d} on mu(k).
#pragma once

#include "ls_internal.cuh"

struct StripGeom {
    int n, t, E, q;
    double shift_over_omega;  // c / w
};

__host__ __device__ __forceinline__ double strip_cutoff(const StripGeom& g, int l, int z) {
    int dist;
    if (z < l * g.t) dist = l * g.t - z;
    else if (z >= (l + 1) * g.t) dist = z - (l + 1) * g.t + 1;
    else dist = 0;
    if (dist <= 1) return 1.0;
    const double tau = (double)(dist - 1) / (double)(g.E - 1);
    return 1.0 - 3.0 * tau * tau + 2.0 * tau * tau * tau;
}

// Coefficient of C^l coupling unknown (r, i) to (r + dz, i + dx) in layer l.
// tab: stencil tables of this direction's grid; m: its medium (n x n, x fastest).
__device__ __forceinline__ double2 strip_coef(const StripGeom& g, const StencilTables* __restrict__ tab,
                                              const double* __restrict__ m, int l, int r, int i, int dx, int dz) {
    const int z0 = l * g.t - g.E;
    const int z = z0 + r;
    if (z < 0 || z >= g.n) return (dx == 0 && dz == 0) ? make_double2(1.0, 0.0) : make_double2(0.0, 0.0);
    if (i + dx < 0 || i + dx >= g.n) return make_double2(0.0, 0.0);
    const int r_lo = z0 < 0 ? -z0 : 0;
    const int r_hi = (z0 + g.q - 1 >= g.n) ? (g.n - 1 - z0) : (g.q - 1);
    const int bz = r == r_lo ? -1 : (r == r_hi ? 1 : 0);
    const int bx = i == 0 ? -1 : (i == g.n - 1 ? 1 : 0);
    if ((bz == -1 && dz == -1) || (bz == 1 && dz == 1)) return make_double2(0.0, 0.0);
    if ((bx == -1 && dx == -1) || (bx == 1 && dx == 1)) return make_double2(0.0, 0.0);
    const int t9 = (bz + 1) * 3 + (bx + 1), s = (dz + 1) * 3 + (dx + 1);
    const double2 a = tab->alpha[t9 * 9 + s];
    const double2 b = tab->wbeta[t9 * 9 + s];
    const int zz = z + dz;
    const double xi = strip_cutoff(g, l, zz);
    // m^l = xi m + i (c/w)(1 - xi)
    const double2 ml = make_double2(xi * m[(size_t)zz * g.n + (i + dx)], g.shift_over_omega * (1.0 - xi));
    return a + b * ml;
}
