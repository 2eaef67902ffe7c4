/*
 * aniso_oracle.c -- plain, slow, FP64 CPU oracle for the directionally split
 * semi-implicit anisotropic-diffusion step of Sharma & Hammett, "A Fast
 * Semi-implicit Method for Anisotropic Diffusion" (arXiv:1008.0861).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  The GPU library never links,
 * calls or includes anything from this directory, and this file includes
 * nothing from the GPU library.
 *
 * What it computes (Section 2 of the paper):
 *   dT/dt = -div q,  q = -chi_par b (b . grad T)                 (Eqs. 1-2)
 * split into an x-update (Eq. xup) and a y-update (Eq. yup).  Each update
 * treats the face-normal part of the flux implicitly, which gives one
 * tridiagonal system per grid line, and the transverse part explicitly with
 * limited face differences (the two DeltaT-bar equations after Eq. yup).
 * The operator form of one step is Eq. op_2step.
 *
 * Readings where the paper is silent:
 *  - b is averaged to faces by the plain mean of the two adjacent cell
 *    centres (Section 2, text after Eq. yup); the implicit coefficient is the
 *    square of the averaged component, as Eq. xup writes it.
 *  - chi_perp (the general SPD tensor of Section 2.1) enters as
 *    D = chi_perp I + (chi_par - chi_perp) b b^T; coefficients are stored in
 *    units of chi_par: kappa = chi_perp/chi_par,
 *      cxx = kappa + (1-kappa) bx^2,  cxy = (1-kappa) bx by   (x faces)
 *      cyy = kappa + (1-kappa) by^2,  cyx = (1-kappa) by bx   (y faces)
 *  - zero-flux ("reflective", Section 3.1) boundaries: the whole flux through
 *    a boundary face is zero, and a ghost cell mirrors its neighbour, so a
 *    limited difference that reaches outside the grid is zero.
 *  - periodic boundaries wrap; the line systems are then cyclic.
 *  - face i+1/2 of row j is stored at [j][i]; face j+1/2 of column i at
 *    [j][i].  Under zero-flux the last face of each line (the boundary face)
 *    is stored as zero.
 *  - update order: Eq. op_2step applies the x-update and then the
 *    y-update in every step; the reversed order is also offered, as the
 *    paper says results barely depend on it (Section 2).  A third option
 *    alternates the two orders from step to step (x,y,y,x,x,y,...).  The
 *    paper does not use it, and it pairs the updates like the Strang
 *    splitting that Section 2 reports as unstable for large timesteps.
 *
 * Arithmetic is IEEE FP64 with no contraction (built with -ffp-contract=off)
 * so the x86 host and the Arm host give identical bits.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_BC_ZEROFLUX 0
#define OR_BC_PERIODIC 1
#define OR_BC_DIRICHLET 2 /* boundary nodes hold their values (T fixed at the domain edge) */

#define OR_LIM_VANLEER 0
#define OR_LIM_ARITH 1 /* arithmetic mean: the linear-analysis reading of Section 2.1 */
#define OR_LIM_MINMOD 2
#define OR_LIM_MC 3

#define OR_ORDER_XY 0        /* Eq. op_2step: x-update, then y-update */
#define OR_ORDER_YX 1        /* the reversed order (text after Eq. op_2step) */
#define OR_ORDER_ALTERNATE 2 /* x then y on even step counters, y then x on odd */

/* ---------------------------------------------------------------- limiters */

/* Two-argument limiters.  van Leer is Eq. vanLeer: 2ab/(a+b) when a and b
 * have the same strict sign, else 0.  The sign test is written on the signs,
 * not on the product, so that tiny differences do not underflow to zero. */
static int same_sign(double a, double b) { return (a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0); }

static double lim2(int lim, double a, double b)
{
    if (lim == OR_LIM_VANLEER) {
        if (!same_sign(a, b)) return 0.0;
        return 2.0 * a * b / (a + b);
    }
    if (lim == OR_LIM_MINMOD) {
        if (!same_sign(a, b)) return 0.0;
        return (a > 0.0) ? fmin(a, b) : fmax(a, b);
    }
    if (lim == OR_LIM_MC) {
        /* monotonized central: sign * min(2|a|, 2|b|, |a+b|/2) */
        if (!same_sign(a, b)) return 0.0;
        double m = fmin(fmin(2.0 * fabs(a), 2.0 * fabs(b)), 0.5 * fabs(a + b));
        return (a > 0.0) ? m : -m;
    }
    return 0.5 * (a + b);
}

/* L(a,b,c,d) = L(L(a,b), L(c,d)), the nesting stated after Eq. vanLeer. */
double or_limit4(int lim, double a, double b, double c, double d)
{
    if (lim == OR_LIM_ARITH) return 0.25 * (a + b + c + d);
    return lim2(lim, lim2(lim, a, b), lim2(lim, c, d));
}

/* ------------------------------------------------------ face coefficients */

/* Cell-centred unit field b -> face coefficients (Section 2: the unit vector
 * at a face is the plain mean of its two neighbouring cell centres).  Arrays
 * are [ny][nx], row-major, x fastest. */
void or_face_coeffs(int nx, int ny, int bc, double kappa, const double *bx, const double *by,
                    double *cxx, double *cxy, double *cyy, double *cyx)
{
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            size_t o = (size_t)j * nx + i;
            /* x face i+1/2 between cells (i,j) and (i+1,j) */
            if (bc == OR_BC_ZEROFLUX && i == nx - 1) {
                cxx[o] = 0.0;
                cxy[o] = 0.0;
            } else {
                int i1 = (i + 1) % nx;
                size_t o1 = (size_t)j * nx + i1;
                double fbx = 0.5 * (bx[o] + bx[o1]);
                double fby = 0.5 * (by[o] + by[o1]);
                cxx[o] = kappa + (1.0 - kappa) * (fbx * fbx);
                cxy[o] = (1.0 - kappa) * (fbx * fby);
            }
            /* y face j+1/2 between cells (i,j) and (i,j+1) */
            if (bc == OR_BC_ZEROFLUX && j == ny - 1) {
                cyy[o] = 0.0;
                cyx[o] = 0.0;
            } else {
                int j1 = (j + 1) % ny;
                size_t o1 = (size_t)j1 * nx + i;
                double fbx = 0.5 * (bx[o] + bx[o1]);
                double fby = 0.5 * (by[o] + by[o1]);
                cyy[o] = kappa + (1.0 - kappa) * (fby * fby);
                cyx[o] = (1.0 - kappa) * (fby * fbx);
            }
        }
    }
}

/* ------------------------------------------------------ tridiagonal solves */

/* Thomas algorithm for a_k x_{k-1} + b_k x_k + c_k x_{k+1} = d_k, k=0..n-1
 * (a_0 and c_{n-1} ignored).  w: scratch of n doubles.  Returns 0, or -1 on
 * a zero pivot. */
int or_thomas(int n, const double *a, const double *b, const double *c, const double *d, double *x,
              double *w)
{
    if (n <= 0) return 0;
    double den = b[0];
    if (den == 0.0) return -1;
    w[0] = c[0] / den;
    x[0] = d[0] / den;
    for (int k = 1; k < n; ++k) {
        den = b[k] - a[k] * w[k - 1];
        if (den == 0.0) return -1;
        w[k] = (k < n - 1) ? c[k] / den : 0.0;
        x[k] = (d[k] - a[k] * x[k - 1]) / den;
    }
    for (int k = n - 2; k >= 0; --k) x[k] = x[k] - w[k] * x[k + 1];
    return 0;
}

/* Cyclic tridiagonal solve: as above but a_0 couples x_{n-1} and c_{n-1}
 * couples x_0.  Sherman-Morrison: A = A' + u v^T with A' tridiagonal,
 * u = (g, 0..0, c_{n-1}), v = (1, 0..0, a_0/g), g = -b_0.  Then
 * x = y - (v.y)/(1 + v.z) z with A'y = d, A'z = u.  w: scratch 4n. */
int or_cyclic(int n, const double *a, const double *b, const double *c, const double *d, double *x,
              double *w)
{
    if (n == 1) {
        double s = a[0] + b[0] + c[0];
        if (s == 0.0) return -1;
        x[0] = d[0] / s;
        return 0;
    }
    if (n == 2) {
        /* both off-diagonal couplings of each row land on the other unknown */
        double m00 = b[0], m01 = a[0] + c[0], m10 = a[1] + c[1], m11 = b[1];
        double det = m00 * m11 - m01 * m10;
        if (det == 0.0) return -1;
        x[0] = (d[0] * m11 - m01 * d[1]) / det;
        x[1] = (m00 * d[1] - m10 * d[0]) / det;
        return 0;
    }
    double *bb = w, *u = w + n, *z = w + 2 * n, *tw = w + 3 * n;
    double g = -b[0];
    if (g == 0.0) return -1;
    for (int k = 0; k < n; ++k) { bb[k] = b[k]; u[k] = 0.0; }
    bb[0] = b[0] - g;
    bb[n - 1] = b[n - 1] - a[0] * c[n - 1] / g;
    u[0] = g;
    u[n - 1] = c[n - 1];
    if (or_thomas(n, a, bb, c, d, x, tw)) return -1;
    if (or_thomas(n, a, bb, c, u, z, tw)) return -1;
    double vy = x[0] + a[0] / g * x[n - 1];
    double vz = z[0] + a[0] / g * z[n - 1];
    double f = vy / (1.0 + vz);
    for (int k = 0; k < n; ++k) x[k] -= f * z[k];
    return 0;
}

/* --------------------------------------------------------------- x-update */

/* Eq. xup for one row j.  Tm, T0, Tp: rows j-1, j, j+1 of T^n (the caller
 * passes T0 for a mirrored ghost row).  cxx_row, cxy_row: x-face coefficients
 * of row j (face i+1/2 at index i).  lamx = chi dt/dx^2, mu = chi dt/(dx dy).
 * out: T* of row j.  w: scratch of 9*nx doubles. */
void or_xsweep_row(int nx, int mode, const double *Tm, const double *T0, const double *Tp,
                   const double *cxx_row, const double *cxy_row, double lamx, double mu, int lim,
                   double *out, double *w)
{
    /* mode: OR_BC_ZEROFLUX, OR_BC_PERIODIC, or OR_BC_DIRICHLET (the first and
     * last cell keep their values: identity rows) */
    int periodic = mode == OR_BC_PERIODIC, pinned = mode == OR_BC_DIRICHLET;
    double *flux = w;          /* transverse term at face i+1/2 (index i)  */
    double *a = w + nx, *b = w + 2 * nx, *c = w + 3 * nx, *d = w + 4 * nx;
    double *tw = w + 5 * nx;   /* 4*nx for the cyclic solver */

    for (int i = 0; i < nx; ++i) {
        int boundary = (!periodic && i == nx - 1);
        if (boundary) { flux[i] = 0.0; continue; }
        int ip = (i + 1) % nx;
        /* DeltaT-bar at x face (i+1/2, j): limited y-differences of cells
         * i+1 and i (first DeltaT-bar equation after Eq. yup). */
        double dT = or_limit4(lim, Tp[ip] - T0[ip], T0[ip] - Tm[ip], Tp[i] - T0[i], T0[i] - Tm[i]);
        flux[i] = cxy_row[i] * dT;
    }
    for (int i = 0; i < nx; ++i) {
        double fplus = flux[i];
        double fminus;
        if (i == 0) fminus = periodic ? flux[nx - 1] : 0.0;
        else fminus = flux[i - 1];
        /* implicit normal part: b_x^2 at faces i+1/2 and i-1/2 */
        double cp = cxx_row[i];
        double cm;
        if (i == 0) cm = periodic ? cxx_row[nx - 1] : 0.0;
        else cm = cxx_row[i - 1];
        if (!periodic && i == nx - 1) cp = 0.0;
        a[i] = -lamx * cm;
        c[i] = -lamx * cp;
        b[i] = 1.0 + lamx * (cm + cp);
        d[i] = T0[i] + mu * (fplus - fminus);
    }
    if (pinned) {
        a[0] = c[0] = a[nx - 1] = c[nx - 1] = 0.0;
        b[0] = b[nx - 1] = 1.0;
        d[0] = T0[0];
        d[nx - 1] = T0[nx - 1];
    }
    if (periodic) or_cyclic(nx, a, b, c, d, out, tw);
    else or_thomas(nx, a, b, c, d, out, tw);
}

/* --------------------------------------------------------------- y-update */

/* Eq. yup for one column i.  Tl, T0, Tr: columns i-1, i, i+1 of T* stored
 * contiguously (index j).  cyy_col, cyx_col: y-face coefficients of column i
 * (face j+1/2 at index j).  lamy = chi dt/dy^2.  out: T^{n+1} of column i. */
void or_ysweep_col(int ny, int mode, const double *Tl, const double *T0, const double *Tr,
                   const double *cyy_col, const double *cyx_col, double lamy, double mu, int lim,
                   double *out, double *w)
{
    int periodic = mode == OR_BC_PERIODIC, pinned = mode == OR_BC_DIRICHLET;
    double *flux = w;
    double *a = w + ny, *b = w + 2 * ny, *c = w + 3 * ny, *d = w + 4 * ny;
    double *tw = w + 5 * ny;

    for (int j = 0; j < ny; ++j) {
        int boundary = (!periodic && j == ny - 1);
        if (boundary) { flux[j] = 0.0; continue; }
        int jp = (j + 1) % ny;
        /* DeltaT-bar at y face (i, j+1/2): limited x-differences of rows
         * j+1 and j (second DeltaT-bar equation after Eq. yup). */
        double dT = or_limit4(lim, Tr[jp] - T0[jp], T0[jp] - Tl[jp], Tr[j] - T0[j], T0[j] - Tl[j]);
        flux[j] = cyx_col[j] * dT;
    }
    for (int j = 0; j < ny; ++j) {
        double fplus = flux[j];
        double fminus;
        if (j == 0) fminus = periodic ? flux[ny - 1] : 0.0;
        else fminus = flux[j - 1];
        double cp = cyy_col[j];
        double cm;
        if (j == 0) cm = periodic ? cyy_col[ny - 1] : 0.0;
        else cm = cyy_col[j - 1];
        if (!periodic && j == ny - 1) cp = 0.0;
        a[j] = -lamy * cm;
        c[j] = -lamy * cp;
        b[j] = 1.0 + lamy * (cm + cp);
        d[j] = T0[j] + mu * (fplus - fminus);
    }
    if (pinned) {
        a[0] = c[0] = a[ny - 1] = c[ny - 1] = 0.0;
        b[0] = b[ny - 1] = 1.0;
        d[0] = T0[0];
        d[ny - 1] = T0[ny - 1];
    }
    if (periodic) or_cyclic(ny, a, b, c, d, out, tw);
    else or_thomas(ny, a, b, c, d, out, tw);
}

/* ------------------------------------------------------------ full sweeps */

/* x-update of the whole grid: rows are independent (OpenMP over rows; the
 * result does not depend on the thread count). */
void or_xsweep(int nx, int ny, int bc, const double *cxx, const double *cxy, double lamx, double mu,
               int lim, const double *Tin, double *Tout)
{
    int periodic = (bc == OR_BC_PERIODIC);
#pragma omp parallel
    {
        double *w = (double *)malloc(sizeof(double) * 9 * (size_t)nx);
#pragma omp for schedule(static)
        for (int j = 0; j < ny; ++j) {
            if (bc == OR_BC_DIRICHLET && (j == 0 || j == ny - 1)) {  /* boundary row: fixed */
                memcpy(Tout + (size_t)j * nx, Tin + (size_t)j * nx, sizeof(double) * (size_t)nx);
                continue;
            }
            int jm = j - 1, jp = j + 1;
            if (jm < 0) jm = periodic ? ny - 1 : 0;      /* mirrored ghost row */
            if (jp >= ny) jp = periodic ? 0 : ny - 1;
            or_xsweep_row(nx, bc, Tin + (size_t)jm * nx, Tin + (size_t)j * nx,
                          Tin + (size_t)jp * nx, cxx + (size_t)j * nx, cxy + (size_t)j * nx, lamx,
                          mu, lim, Tout + (size_t)j * nx, w);
        }
        free(w);
    }
}

/* y-update of the whole grid: columns are gathered into contiguous buffers. */
void or_ysweep(int nx, int ny, int bc, const double *cyy, const double *cyx, double lamy, double mu,
               int lim, const double *Tin, double *Tout)
{
    int periodic = (bc == OR_BC_PERIODIC);
#pragma omp parallel
    {
        double *buf = (double *)malloc(sizeof(double) * 15 * (size_t)ny);
        double *Tl = buf, *T0 = buf + ny, *Tr = buf + 2 * ny, *gy = buf + 3 * ny,
               *ey = buf + 4 * ny, *o = buf + 5 * ny, *w = buf + 6 * ny;
#pragma omp for schedule(static)
        for (int i = 0; i < nx; ++i) {
            if (bc == OR_BC_DIRICHLET && (i == 0 || i == nx - 1)) {  /* boundary column: fixed */
                for (int j = 0; j < ny; ++j) Tout[(size_t)j * nx + i] = Tin[(size_t)j * nx + i];
                continue;
            }
            int il = i - 1, ir = i + 1;
            if (il < 0) il = periodic ? nx - 1 : 0;      /* mirrored ghost column */
            if (ir >= nx) ir = periodic ? 0 : nx - 1;
            for (int j = 0; j < ny; ++j) {
                size_t r = (size_t)j * nx;
                Tl[j] = Tin[r + il];
                T0[j] = Tin[r + i];
                Tr[j] = Tin[r + ir];
                gy[j] = cyy[r + i];
                ey[j] = cyx[r + i];
            }
            or_ysweep_col(ny, bc, Tl, T0, Tr, gy, ey, lamy, mu, lim, o, w);
            for (int j = 0; j < ny; ++j) Tout[(size_t)j * nx + i] = o[j];
        }
        free(buf);
    }
}

/* ------------------------------------------------------------- full steps */

/* nsteps steps of Eq. op_2step, in place on T.  The step counter of the
 * first step is step0; the order of the two updates follows `order`.
 * lamx = chi dt/dx^2, lamy = chi dt/dy^2, mu = chi dt/(dx dy).
 * Returns 0, or -1 if scratch could not be allocated. */
int or_step(int nx, int ny, int bc, const double *cxx, const double *cxy, const double *cyy,
            const double *cyx, double lamx, double lamy, double mu, int lim, int order,
            long long step0, int nsteps, double *T, const double *Q, double dt)
{
    double *Ts = (double *)malloc(sizeof(double) * (size_t)nx * ny);
    if (!Ts) return -1;
    for (int n = 0; n < nsteps; ++n) {
        /* optional source term, applied as an explicit stage before the
         * updates (the convergence test of Section 3.2 adds Q to Eq. 1) */
        if (Q)
            for (size_t k = 0; k < (size_t)nx * ny; ++k) T[k] += dt * Q[k];
        long long s = step0 + n;
        int x_first = (order == OR_ORDER_XY) || (order == OR_ORDER_ALTERNATE && (s % 2) == 0);
        if (x_first) {
            or_xsweep(nx, ny, bc, cxx, cxy, lamx, mu, lim, T, Ts);
            or_ysweep(nx, ny, bc, cyy, cyx, lamy, mu, lim, Ts, T);
        } else {
            or_ysweep(nx, ny, bc, cyy, cyx, lamy, mu, lim, T, Ts);
            or_xsweep(nx, ny, bc, cxx, cxy, lamx, mu, lim, Ts, T);
        }
    }
    free(Ts);
    return 0;
}

/* ------------------------------------------- temperature-dependent chi */

/* Section 3.3 runs the method with chi_par proportional to T^(5/2), the
 * diffusivity taken at each face from the current temperature by a harmonic
 * average of the two cells beside it (the interpolation the paper's earlier
 * work prescribes, Section 2).  Readings: chi(T) = chi_par (max(T,0)/t_ref)^alpha;
 * "current" is the input of each directional update (T^n for the x-update,
 * T* for the y-update), so each update stays linear in its unknown; the face
 * factor multiplies the normal and the transverse coefficient alike (and so
 * chi_perp scales with chi_par). */
static double chi_ratio(double T, double alpha, double t_ref)
{
    return T > 0.0 ? pow(T / t_ref, alpha) : 0.0;
}

static double harmonic(double a, double b)
{
    return (a > 0.0 && b > 0.0) ? 2.0 * a * b / (a + b) : 0.0;
}

/* Face coefficients of one update scaled by the face factor of T: axis 0
 * scales cxx, cxy at x faces (cells (i,j), (i+1,j)); axis 1 scales cyy, cyx
 * at y faces (cells (i,j), (i,j+1)).  The neighbour index wraps; zero-flux
 * boundary faces keep their zero coefficients. */
void or_nl_coeffs(int nx, int ny, int axis, double alpha, double t_ref, const double *cn, const double *ct,
                  const double *T, double *gn, double *gt)
{
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const size_t o = (size_t)j * nx + i;
            const size_t o1 = axis == 0 ? (size_t)j * nx + (i + 1) % nx : (size_t)((j + 1) % ny) * nx + i;
            const double h = harmonic(chi_ratio(T[o], alpha, t_ref), chi_ratio(T[o1], alpha, t_ref));
            gn[o] = cn[o] * h;
            gt[o] = ct[o] * h;
        }
}

/* nsteps x-then-y steps (Eq. op_2step) in place on T with the face factor
 * recomputed from each update's input.  Returns 0, or -1 on allocation
 * failure. */
int or_step_nl(int nx, int ny, int bc, const double *cxx, const double *cxy, const double *cyy,
               const double *cyx, double lamx, double lamy, double mu, int lim, double alpha, double t_ref,
               int nsteps, double *T)
{
    const size_t n = (size_t)nx * ny;
    double *Ts = (double *)malloc(sizeof(double) * n);
    double *g = (double *)malloc(sizeof(double) * n);
    double *e = (double *)malloc(sizeof(double) * n);
    if (!Ts || !g || !e) {
        free(Ts);
        free(g);
        free(e);
        return -1;
    }
    for (int s = 0; s < nsteps; ++s) {
        or_nl_coeffs(nx, ny, 0, alpha, t_ref, cxx, cxy, T, g, e);
        or_xsweep(nx, ny, bc, g, e, lamx, mu, lim, T, Ts);
        or_nl_coeffs(nx, ny, 1, alpha, t_ref, cyy, cyx, Ts, g, e);
        or_ysweep(nx, ny, bc, g, e, lamy, mu, lim, Ts, T);
    }
    free(Ts);
    free(g);
    free(e);
    return 0;
}

/* ------------------------------------------------ explicit limited step */

/* Flux through x face (i+1/2, j) of the explicit step: the normal part of
 * Eq. xup and its limited transverse part, both from T.  Zero through a
 * zero-flux boundary face; rows outside the grid are mirrored (zero-flux) or
 * wrapped (periodic), as in the sweeps. */
static double ex_fx(int nx, int ny, int per, const double *cxx, const double *cxy, double lamx,
                    double mu, int lim, const double *T, int i, int j)
{
    if (!per && i == nx - 1) return 0.0;
    int ip = (i + 1) % nx;
    int jm = j - 1, jp = j + 1;
    if (jm < 0) jm = per ? ny - 1 : 0;
    if (jp >= ny) jp = per ? 0 : ny - 1;
    const double *rm = T + (size_t)jm * nx, *r0 = T + (size_t)j * nx, *rp = T + (size_t)jp * nx;
    double dT = or_limit4(lim, rp[ip] - r0[ip], r0[ip] - rm[ip], rp[i] - r0[i], r0[i] - rm[i]);
    return lamx * cxx[(size_t)j * nx + i] * (r0[ip] - r0[i]) + mu * cxy[(size_t)j * nx + i] * dT;
}

/* Flux through y face (i, j+1/2) (second DeltaT-bar equation after Eq. yup). */
static double ex_fy(int nx, int ny, int per, const double *cyy, const double *cyx, double lamy,
                    double mu, int lim, const double *T, int i, int j)
{
    if (!per && j == ny - 1) return 0.0;
    int jp = (j + 1) % ny;
    int im = i - 1, ip = i + 1;
    if (im < 0) im = per ? nx - 1 : 0;
    if (ip >= nx) ip = per ? 0 : nx - 1;
    const double *r0 = T + (size_t)j * nx, *r1 = T + (size_t)jp * nx;
    double dT = or_limit4(lim, r1[ip] - r1[i], r1[i] - r1[im], r0[ip] - r0[i], r0[i] - r0[im]);
    return lamy * cyy[(size_t)j * nx + i] * (r1[i] - r0[i]) + mu * cyx[(size_t)j * nx + i] * dT;
}

/* nsteps steps of the explicit limited scheme, in place on T: the unsplit
 * explicit form of the face fluxes of Eqs. xup and yup, every flux taken at
 * T^n (the explicit method the paper compares against, Sections 1 and 3.1):
 *   T^{n+1}_ij = T^n_ij + Fx(i+1/2,j) - Fx(i-1/2,j) + Fy(i,j+1/2) - Fy(i,j-1/2).
 * Returns 0, or -1 if scratch could not be allocated. */
int or_explicit_step(int nx, int ny, int bc, const double *cxx, const double *cxy, const double *cyy,
                     const double *cyx, double lamx, double lamy, double mu, int lim, int nsteps,
                     double *T)
{
    int per = bc == OR_BC_PERIODIC;
    double *Tn = (double *)malloc(sizeof(double) * (size_t)nx * ny);
    if (!Tn) return -1;
    for (int n = 0; n < nsteps; ++n) {
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                double fxp = ex_fx(nx, ny, per, cxx, cxy, lamx, mu, lim, T, i, j);
                double fxm = i > 0 ? ex_fx(nx, ny, per, cxx, cxy, lamx, mu, lim, T, i - 1, j)
                                   : (per ? ex_fx(nx, ny, per, cxx, cxy, lamx, mu, lim, T, nx - 1, j) : 0.0);
                double fyp = ex_fy(nx, ny, per, cyy, cyx, lamy, mu, lim, T, i, j);
                double fym = j > 0 ? ex_fy(nx, ny, per, cyy, cyx, lamy, mu, lim, T, i, j - 1)
                                   : (per ? ex_fy(nx, ny, per, cyy, cyx, lamy, mu, lim, T, i, ny - 1) : 0.0);
                Tn[(size_t)j * nx + i] = T[(size_t)j * nx + i] + (fxp - fxm) + (fyp - fym);
                if (bc == OR_BC_DIRICHLET && (i == 0 || j == 0 || i == nx - 1 || j == ny - 1))
                    Tn[(size_t)j * nx + i] = T[(size_t)j * nx + i];  /* boundary node: fixed */
            }
        }
        memcpy(T, Tn, sizeof(double) * (size_t)nx * ny);
    }
    free(Tn);
    return 0;
}

/* FP64 sum (plain left-to-right), minimum and maximum of n values. */
void or_totals(size_t n, const double *T, double *sum, double *tmin, double *tmax)
{
    double s = 0.0, lo = INFINITY, hi = -INFINITY;
    for (size_t k = 0; k < n; ++k) {
        s += T[k];
        if (T[k] < lo) lo = T[k];
        if (T[k] > hi) hi = T[k];
    }
    *sum = s;
    *tmin = lo;
    *tmax = hi;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the number of OpenMP threads the oracle uses (results do not depend
 * on it: every line is solved independently). */
void or_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
