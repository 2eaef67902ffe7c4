// explicit_kernel.cuh -- explicit limited step: the face fluxes of Eqs. xup
// and yup (normal part and limited transverse part) all evaluated at T^n and
// applied explicitly,
//   T^{n+1}_ij = T^n_ij + Fx(i+1/2,j) - Fx(i-1/2,j) + Fy(i,j+1/2) - Fy(i,j-1/2),
// the explicit method the paper measures its speed-up against (Sections 1
// and 3.1).  Stable for dt up to about the explicit limit.
//
// A thread owns one column i of a strip of rows and walks down it: row j+1
// is loaded once, columns i-1 and i+1 come from the neighbouring lanes
// (lanes at a tile edge load their outside neighbour), and the y-face flux
// below row j is the one computed above row j-1.  Limited differences nest
// as in Eq. vanLeer: an inner value per cell and direction, then one per
// face.  Ghost rows and columns are mirrored (zero-flux) or wrapped
// (periodic); zero-flux boundary faces carry zero coefficients.
#pragma once
#include "line4_kernel.cuh"

namespace aniso {

template <typename R, typename C, bool VL>
__global__ void __launch_bounds__(256) explicit_kernel(ExpArgs a)
{
    const int nx = a.nx, ny = a.ny, per = a.per, lim = a.limiter;
    const int lane = threadIdx.x;  // blockDim.x == 32
    const int i = blockIdx.x * 32 + lane;
    const int j0 = (blockIdx.y * blockDim.y + threadIdx.y) * a.rows;
    const bool col_ok = i < nx;
    const unsigned full = 0xffffffffu;
    if (j0 >= ny) return;  // whole warp: j0 is uniform across it
    const int j1 = min(j0 + a.rows, ny);
    auto cw = [&](int c) { return per ? (c + nx) % nx : (c < 0 ? 0 : (c >= nx ? nx - 1 : c)); };
    auto rw = [&](int r) { return per ? (r + ny) % ny : (r < 0 ? 0 : (r >= ny ? ny - 1 : r)); };
    const int ic = col_ok ? i : nx - 1;
    const int il = cw(ic - 1), ir = cw(ic + 1);
    const R *T = static_cast<const R *>(a.Tin);
    const C *cxx = static_cast<const C *>(a.cxx), *cxy = static_cast<const C *>(a.cxy);
    const C *cyy = static_cast<const C *>(a.cyy), *cyx = static_cast<const C *>(a.cyx);
    const R lamx = (R)a.lamx, lamy = (R)a.lamy, mu = (R)a.mu;
    R *out = static_cast<R *>(a.Tout);
    bool bad = false;

    // values of column i and its two neighbours on one row
    struct Row {
        R l, c, r;
    };
    auto load_row = [&](int r) {
        const R *p = T + (size_t)rw(r) * nx;
        Row v;
        v.c = p[ic];
        R fromL = __shfl_up_sync(full, v.c, 1), fromR = __shfl_down_sync(full, v.c, 1);
        v.l = (lane == 0 || !col_ok || ic - 1 < 0 || i - 1 >= nx) ? p[il] : fromL;
        v.r = (lane == 31 || i + 1 >= nx) ? p[ir] : fromR;
        return v;
    };
    // x-face flux at face (col)+1/2 of row j from rows jm, j, jp (columns col, col+1)
    auto fx = [&](int col, int j, R Tm0, R T0, R Tp0, R Tm1, R T1, R Tp1) {
        const size_t o = (size_t)j * nx + col;
        const R v0 = level<R, VL>(lim, Tp0 - T0, T0 - Tm0), v1 = level<R, VL>(lim, Tp1 - T1, T1 - Tm1);
        return lamx * (R)ldcoef(cxx + o) * (T1 - T0) + mu * (R)ldcoef(cxy + o) * level<R, VL>(lim, v1, v0);
    };
    // y-face flux at face j+1/2 of column i from rows j (a) and j+1 (b)
    auto fy = [&](int j, const Row &ra, const Row &rb) {
        const size_t o = (size_t)j * nx + ic;
        const R va = level<R, VL>(lim, ra.r - ra.c, ra.c - ra.l), vb = level<R, VL>(lim, rb.r - rb.c, rb.c - rb.l);
        return lamy * (R)ldcoef(cyy + o) * (rb.c - ra.c) + mu * (R)ldcoef(cyx + o) * level<R, VL>(lim, vb, va);
    };

    Row rm = load_row(j0 - 1), rc = load_row(j0);
    // flux through the face below the strip (zero-flux: zero coefficients there)
    R Fym = fy(rw(j0 - 1), rm, rc);
    if (!per && j0 == 0) Fym = R(0);
    for (int j = j0; j < j1; ++j) {
        const Row rp = load_row(j + 1);
        // x faces i+1/2 and i-1/2 of row j
        const R Fxp = fx(ic, j, rm.c, rc.c, rp.c, rm.r, rc.r, rp.r);
        R Fxm = __shfl_up_sync(full, Fxp, 1);
        if (lane == 0 || !col_ok) Fxm = fx(il, j, rm.l, rc.l, rp.l, rm.c, rc.c, rp.c);
        if (!per && ic == 0) Fxm = R(0);
        const R Fyp = fy(j, rc, rp);
        R Tn = rc.c + (Fxp - Fxm) + (Fyp - Fym);
        if (a.pin && (i == 0 || i == nx - 1 || j == 0 || j == ny - 1)) Tn = rc.c;  // fixed boundary node
        if (col_ok) {
            out[(size_t)j * nx + i] = Tn;
            bad |= !(fabs(Tn) < R(INFINITY));
        }
        Fym = Fyp;
        rm = rc;
        rc = rp;
    }
    if (bad) atomicOr(a.err, 1u);
}

}  // namespace aniso
