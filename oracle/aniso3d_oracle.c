/*
 * aniso3d_oracle.c -- plain, slow, FP64 CPU oracle for the three-dimensional
 * form of the split semi-implicit step (Sharma & Hammett, arXiv:1008.0861,
 * Section 2.1: the 3-D amplification factor r1 r2 r3 and its stability
 * limit; Section 2 states that the extension to three dimensions follows
 * the two-dimensional one directly).
 *
 * THIS IS TEST INFRASTRUCTURE, like aniso_oracle.c (which supplies the
 * limiter and the two line solvers used here).  The GPU library never links,
 * calls or includes anything from this directory.
 *
 * What it computes.  Each step applies three directional updates in the
 * order x, y, z; each is Eq. xup with one more transverse term.  For the
 * update along axis d with transverse axes a and b, at face f+1/2 of a line:
 *   F_{f+1/2} = mu_da c_da DeltaT-bar^a_{f+1/2} + mu_db c_db DeltaT-bar^b_{f+1/2}
 * where DeltaT-bar^a is the nested limited difference of the paper (the
 * a-differences of the two cells beside the face, limited per cell, then
 * limited together), and the line system is
 *   -lam c_dd[f-1] T'_{f-1} + (1 + lam (c_dd[f-1] + c_dd[f])) T'_f
 *       - lam c_dd[f] T'_{f+1} = T_f + F_{f+1/2} - F_{f-1/2},
 * lam = chi dt / Delta_d^2, mu_da = chi dt / (Delta_d Delta_a).  With constant
 * b and the arithmetic-mean limiter a Fourier mode is multiplied by the
 * paper's r1 (and its two analogues) in the three updates.
 *
 * Readings where the paper is silent:
 *  - coefficients: D = chi_perp I + (chi_par - chi_perp) b b^T in units of
 *    chi_par (kappa = chi_perp / chi_par); at an x face
 *      cxx = kappa + (1-kappa) bx^2,  cxy = (1-kappa) bx by,  cxz = (1-kappa) bx bz
 *    with b averaged to the face from the two adjacent cell centres; the y
 *    and z faces alike (cyy, cyz, cyx; czz, czx, czy).
 *  - boundaries as in two dimensions: zero-flux faces carry zero
 *    coefficients and ghost cells mirror their neighbour; periodic wraps.
 *  - the 4-step scheme (Eq. 4step) in three dimensions: per axis, one
 *    update with the transverse terms and half the implicit coefficient,
 *    then one purely implicit update with half the coefficient (six line
 *    solves per step), axes in the order x, y, z.
 *  - arrays are [nz][ny][nx], x fastest; face f+1/2 along axis d of a cell is
 *    stored at that cell; the boundary face of a zero-flux line is zero.
 *
 * Arithmetic is IEEE FP64 with no contraction (-ffp-contract=off).
 */
#include <stdlib.h>
#include <string.h>

#define OR3_BC_ZEROFLUX 0
#define OR3_BC_PERIODIC 1

double or_limit4(int lim, double a, double b, double c, double d);
int or_thomas(int n, const double *a, const double *b, const double *c, const double *d, double *x,
              double *w);
int or_cyclic(int n, const double *a, const double *b, const double *c, const double *d, double *x,
              double *w);

/* ------------------------------------------------------ face coefficients */

/* Cell-centred unit field (bx, by, bz) -> the nine face coefficients.
 * c[0..2] = cxx, cxy, cxz (x faces); c[3..5] = cyy, cyz, cyx (y faces);
 * c[6..8] = czz, czx, czy (z faces).  In each triple the first is the
 * normal coefficient, the second pairs with the next axis (cyclically) and
 * the third with the one after it. */
void or3_face_coeffs(int nx, int ny, int nz, int bc, double kappa, const double *bx,
                     const double *by, const double *bz, double *const c[9])
{
    const int n3[3] = {nx, ny, nz};
    const size_t st[3] = {1, (size_t)nx, (size_t)nx * ny};
    const double *bv[3] = {bx, by, bz};
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int ix[3] = {i, j, k};
                const size_t o = (size_t)k * st[2] + (size_t)j * st[1] + i;
                for (int d = 0; d < 3; ++d) {
                    const int a = (d + 1) % 3, b = (d + 2) % 3;
                    double *cn = c[3 * d], *ca = c[3 * d + 1], *cb = c[3 * d + 2];
                    if (bc == OR3_BC_ZEROFLUX && ix[d] == n3[d] - 1) {
                        cn[o] = ca[o] = cb[o] = 0.0;
                        continue;
                    }
                    /* neighbour across face ix[d] + 1/2 (wraps when periodic) */
                    const size_t o1 = o - (size_t)ix[d] * st[d] + (size_t)((ix[d] + 1) % n3[d]) * st[d];
                    double fb[3];
                    for (int e = 0; e < 3; ++e) fb[e] = 0.5 * (bv[e][o] + bv[e][o1]);
                    cn[o] = kappa + (1.0 - kappa) * (fb[d] * fb[d]);
                    ca[o] = (1.0 - kappa) * (fb[d] * fb[a]);
                    cb[o] = (1.0 - kappa) * (fb[d] * fb[b]);
                }
            }
}

/* -------------------------------------------------------- one directional update */

/* Update along axis d (0 = x, 1 = y, 2 = z) of the whole grid, Tin -> Tout.
 * cn, ca, cb: the face coefficients of axis d (normal, with axis d+1, with
 * axis d+2, cyclically).  lam = chi dt / Delta_d^2; mua, mub the mixed
 * factors chi dt / (Delta_d Delta_a), chi dt / (Delta_d Delta_b).  Lines
 * are independent (OpenMP over lines; the result does not depend on the
 * thread count). */
void or3_sweep(int nx, int ny, int nz, int bc, int d, const double *cn, const double *ca,
               const double *cb, double lam, double mua, double mub, int lim, const double *Tin,
               double *Tout)
{
    const int n3[3] = {nx, ny, nz};
    const size_t st[3] = {1, (size_t)nx, (size_t)nx * ny};
    const int a = (d + 1) % 3, b = (d + 2) % 3;
    const int n = n3[d], na = n3[a], nb = n3[b];
    const int per = bc == OR3_BC_PERIODIC;
#pragma omp parallel
    {
        double *buf = (double *)malloc(sizeof(double) * 20 * (size_t)n);
        double *T0 = buf, *Tam = buf + n, *Tap = buf + 2 * n, *Tbm = buf + 3 * n, *Tbp = buf + 4 * n;
        double *F = buf + 5 * n, *A = buf + 6 * n, *B = buf + 7 * n, *C = buf + 8 * n, *D = buf + 9 * n;
        double *x = buf + 10 * n, *w = buf + 11 * n; /* w: 4n for the cyclic solver */
#pragma omp for schedule(static)
        for (int line = 0; line < na * nb; ++line) {
            const int ia = line % na, ib = line / na;
            /* neighbouring lines along a and b: wrapped, or mirrored (the line itself) */
            int iam = ia - 1, iap = ia + 1, ibm = ib - 1, ibp = ib + 1;
            if (iam < 0) iam = per ? na - 1 : 0;
            if (iap >= na) iap = per ? 0 : na - 1;
            if (ibm < 0) ibm = per ? nb - 1 : 0;
            if (ibp >= nb) ibp = per ? 0 : nb - 1;
            const size_t base = (size_t)ia * st[a] + (size_t)ib * st[b];
            const size_t bam = (size_t)iam * st[a] + (size_t)ib * st[b];
            const size_t bap = (size_t)iap * st[a] + (size_t)ib * st[b];
            const size_t bbm = (size_t)ia * st[a] + (size_t)ibm * st[b];
            const size_t bbp = (size_t)ia * st[a] + (size_t)ibp * st[b];
            for (int f = 0; f < n; ++f) {
                const size_t s = (size_t)f * st[d];
                T0[f] = Tin[base + s];
                Tam[f] = Tin[bam + s];
                Tap[f] = Tin[bap + s];
                Tbm[f] = Tin[bbm + s];
                Tbp[f] = Tin[bbp + s];
            }
            /* transverse flux at face f+1/2 (limited differences of cells f+1 and f) */
            for (int f = 0; f < n; ++f) {
                if (!per && f == n - 1) {
                    F[f] = 0.0;
                    continue;
                }
                const int g = (f + 1) % n;
                const size_t o = base + (size_t)f * st[d];
                const double dTa = or_limit4(lim, Tap[g] - T0[g], T0[g] - Tam[g], Tap[f] - T0[f], T0[f] - Tam[f]);
                const double dTb = or_limit4(lim, Tbp[g] - T0[g], T0[g] - Tbm[g], Tbp[f] - T0[f], T0[f] - Tbm[f]);
                F[f] = mua * ca[o] * dTa + mub * cb[o] * dTb;
            }
            /* implicit face-normal part */
            for (int f = 0; f < n; ++f) {
                const size_t o = base + (size_t)f * st[d];
                double cp = cn[o], cm, Fm;
                if (f == 0) {
                    cm = per ? cn[base + (size_t)(n - 1) * st[d]] : 0.0;
                    Fm = per ? F[n - 1] : 0.0;
                } else {
                    cm = cn[o - st[d]];
                    Fm = F[f - 1];
                }
                if (!per && f == n - 1) cp = 0.0;
                A[f] = -lam * cm;
                C[f] = -lam * cp;
                B[f] = 1.0 + lam * (cm + cp);
                D[f] = T0[f] + (F[f] - Fm);
            }
            if (per) or_cyclic(n, A, B, C, D, x, w);
            else or_thomas(n, A, B, C, D, x, w);
            for (int f = 0; f < n; ++f) Tout[base + (size_t)f * st[d]] = x[f];
        }
        free(buf);
    }
}

/* ------------------------------------------------------------- full steps */

/* nsteps steps in place on T.  c: the nine face coefficients as
 * or3_face_coeffs orders them.  lam[d] = chi dt / Delta_d^2;
 * mu[d] = { chi dt / (Delta_d Delta_{d+1}), chi dt / (Delta_d Delta_{d+2}) }
 * (axes cyclic) as mu[2d], mu[2d+1].  scheme 0: x, y, z updates (the 2-step
 * scheme of Eq. op_2step with a third factor); scheme 1: the 4-step scheme
 * of Eq. 4step with a third pair of factors.  Returns 0, or -1 if scratch
 * could not be allocated. */
int or3_step(int nx, int ny, int nz, int bc, const double *const c[9], const double lam[3],
             const double mu[6], int lim, int scheme, int nsteps, double *T)
{
    const size_t cells = (size_t)nx * ny * nz;
    double *S = (double *)malloc(sizeof(double) * cells);
    if (!S) return -1;
    for (int s = 0; s < nsteps; ++s) {
        for (int d = 0; d < 3; ++d) {
            const double *cn = c[3 * d], *ca = c[3 * d + 1], *cb = c[3 * d + 2];
            if (scheme == 0) {
                or3_sweep(nx, ny, nz, bc, d, cn, ca, cb, lam[d], mu[2 * d], mu[2 * d + 1], lim, T, S);
                memcpy(T, S, sizeof(double) * cells);
            } else {
                or3_sweep(nx, ny, nz, bc, d, cn, ca, cb, 0.5 * lam[d], mu[2 * d], mu[2 * d + 1], lim, T, S);
                or3_sweep(nx, ny, nz, bc, d, cn, ca, cb, 0.5 * lam[d], 0.0, 0.0, lim, S, T);
            }
        }
    }
    free(S);
    return 0;
}
