// Doubled-lattice stencil geometry shared by the operator kernels (internal).
// Site index s = row * 2L + x, row = (t L + z) L + y (see include/qstar.h).
#pragma once
#include "qs_internal.cuh"

// Coordinates of a doubled site: x in [0, 2L), y, z in [0, L), t in [0, T);
// row = (t L + z) L + y; p = row L + (x mod L) is the physical site.
struct Site {
    int s, x, y, z, t, row, p;
};

__device__ __forceinline__ Site site_of(const Geom &g, int s)
{
    Site c;
    c.s = s;
    c.row = s / g.L2;
    c.x = s - c.row * g.L2;
    int r = c.row;
    c.y = r % g.L;
    r /= g.L;
    c.z = r % g.L;
    c.t = r / g.L;
    c.p = c.row * g.L + (c.x >= g.L ? c.x - g.L : c.x);
    return c;
}

struct Nb {
    int s, p;
    bool mir;
};

// neighbour x + STEP mu (same rules as qs_nbr: x periodic over 2L; crossing y or z
// with C* there also moves x by L; t periodic or antiperiodic)
template <int MU, int STEP>
__device__ __forceinline__ Nb nbr_of(const Geom &g, const Site &c, int *sg)
{
    int x = c.x, row = c.row;
    *sg = 1;
    const int L = g.L, L2 = g.L2;
    if (MU == 0) {
        const int LL = L * L;
        if (STEP > 0) row = (c.t == g.T - 1) ? row - (g.T - 1) * LL : row + LL;
        else row = (c.t == 0) ? row + (g.T - 1) * LL : row - LL;
        if (g.t_anti && ((STEP > 0 && c.t == g.T - 1) || (STEP < 0 && c.t == 0))) *sg = -1;
    } else if (MU == 1) {
        if (STEP > 0) x = (x == L2 - 1) ? 0 : x + 1;
        else x = (x == 0) ? L2 - 1 : x - 1;
    } else {
        const int coord = MU == 2 ? c.y : c.z;
        const int stride = MU == 2 ? 1 : L;
        const int cst = MU == 2 ? g.cstar_y : g.cstar_z;
        bool wrap = STEP > 0 ? (coord == L - 1) : (coord == 0);
        if (wrap) {
            row += STEP > 0 ? -(L - 1) * stride : (L - 1) * stride;
            if (cst) x = x >= L ? x - L : x + L;
        } else {
            row += STEP * stride;
        }
    }
    Nb n;
    n.s = row * L2 + x;
    n.mir = x >= L;
    n.p = row * L + (n.mir ? x - L : x);
    return n;
}

