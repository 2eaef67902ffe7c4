// aniso3d_api.cu -- host side of the three-dimensional split step
// (Section 2.1): handles, validation and the update schedule.
//
// A step is three updates (x, y, z), each implicit in the face-normal flux
// and explicit in the two limited transverse fluxes; the 4-step scheme of
// Eq. 4step takes each axis as two half-coefficient updates, the first
// with the transverse terms.  Every update is one launch of the line kernel
// that writes its result transposed for the next axis (kernels_3d.cu), so
// a 2-step step is three launches: T -> s1 (x), s1 -> s2 (y), s2 -> T (z).
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>

#include "../../include/aniso.h"
#include "aniso_internal.h"
#include "status.h"

using namespace aniso;

struct aniso3_ctx {
    int n[3] = {0, 0, 0};
    double d[3] = {0, 0, 0};
    double chi_par = 0, chi_perp = 0;
    int bc = 0;
    int prec = PREC_FP64, limiter = LIM_VANLEER, scheme = ANISO_SCHEME_2STEP, warps = 0, seg = 0;
    int field_fp16 = 0;  // face coefficients stored as FP16 (FP32 precision only)
    cudaStream_t stream = 0;
    bool field_set = false;
    void *c[9] = {};                    // face coefficients, each axis in its update's layout
    void *s1 = nullptr, *s2 = nullptr;  // intermediates of a step
    double *partials = nullptr, *result = nullptr;
    unsigned *err = nullptr;

    size_t cells() const { return (size_t)n[0] * n[1] * n[2]; }
    size_t esz() const { return prec == PREC_FP64 ? 8 : 4; }
    size_t csz() const { return field_fp16 ? 2 : esz(); }
};

static void free3(aniso3_ctx *h)
{
    for (auto &p : h->c) {
        if (p) cudaFree(p);
        p = nullptr;
    }
    void **bufs[] = {&h->s1, &h->s2, reinterpret_cast<void **>(&h->partials), reinterpret_cast<void **>(&h->result),
                     reinterpret_cast<void **>(&h->err)};
    for (void **b : bufs) {
        if (*b) cudaFree(*b);
        *b = nullptr;
    }
}

// Every axis's lines must fit the line kernel with a transposed output.
static int check_shape(const aniso3_ctx *h, const char *who)
{
    static const char *names = "xyz";
    for (int a = 0; a < 3; ++a) {
        int team, lpb, nt;
        size_t smem;
        if (!line4_config(h->prec, h->n[a], true, h->warps, h->seg, &team, &lpb, &nt, &smem))
            return fail(ANISO_ERR_UNSUPPORTED,
                         "%s: n%c=%d is not a line length the 3-D kernel takes (a multiple of %d, from %d to %d)",
                         who, names[a], h->n[a], h->prec == PREC_FP64 ? 2 : 4, h->prec == PREC_FP64 ? 4 : 8,
                         h->prec == PREC_FP64 ? 1024 : MAX_LINE2_TRANSPOSED);
    }
    return ANISO_OK;
}

extern "C" int aniso3_create(int nx, int ny, int nz, double dx, double dy, double dz, double chi_par, double chi_perp,
                             int bc, aniso3_t *out)
{
    if (!out) return fail(ANISO_ERR_ARG, "aniso3_create: out is NULL");
    *out = nullptr;
    if (nx < 3 || ny < 3 || nz < 3)
        return fail(ANISO_ERR_ARG, "aniso3_create: nx=%d ny=%d nz=%d (need >= 3)", nx, ny, nz);
    if (!(dx > 0) || !(dy > 0) || !(dz > 0)) return fail(ANISO_ERR_ARG, "aniso3_create: dx, dy, dz must be > 0");
    if (!(chi_par > 0)) return fail(ANISO_ERR_ARG, "aniso3_create: chi_par must be > 0");
    if (!(chi_perp >= 0) || chi_perp > chi_par)
        return fail(ANISO_ERR_ARG, "aniso3_create: need 0 <= chi_perp <= chi_par");
    if (bc != ANISO_BC_ZEROFLUX && bc != ANISO_BC_PERIODIC)
        return fail(ANISO_ERR_ARG, "aniso3_create: boundary condition %d (zero-flux or periodic)", bc);
    aniso3_ctx *h = new aniso3_ctx;
    h->n[0] = nx;
    h->n[1] = ny;
    h->n[2] = nz;
    h->d[0] = dx;
    h->d[1] = dy;
    h->d[2] = dz;
    h->chi_par = chi_par;
    h->chi_perp = chi_perp;
    h->bc = bc;
    *out = h;
    return ANISO_OK;
}

extern "C" int aniso3_set_option(aniso3_t h, int key, long long v)
{
    if (!h) return fail(ANISO_ERR_ARG, "aniso3_set_option: null handle");
    switch (key) {
    case ANISO_OPT_PRECISION:
        if (v != ANISO_PREC_FP64 && v != ANISO_PREC_FP32) return fail(ANISO_ERR_ARG, "bad precision %lld", v);
        if (h->field_set && v != h->prec) return fail(ANISO_ERR_STATE, "precision is fixed once the field is set");
        h->prec = (int)v;
        return ANISO_OK;
    case ANISO_OPT_LIMITER:
        if (v < ANISO_LIM_VANLEER || v > ANISO_LIM_MC) return fail(ANISO_ERR_ARG, "bad limiter %lld", v);
        h->limiter = (int)v;
        return ANISO_OK;
    case ANISO_OPT_SCHEME:
        if (v == ANISO_SCHEME_EXPLICIT)
            return fail(ANISO_ERR_UNSUPPORTED, "aniso3_set_option: the explicit scheme is two-dimensional only");
        if (v != ANISO_SCHEME_2STEP && v != ANISO_SCHEME_4STEP) return fail(ANISO_ERR_ARG, "bad scheme %lld", v);
        h->scheme = (int)v;
        return ANISO_OK;
    case ANISO_OPT_STREAM:
        h->stream = reinterpret_cast<cudaStream_t>(v);
        return ANISO_OK;
    case ANISO_OPT_BLOCK_WARPS:
        if (v < 0 || v > 8) return fail(ANISO_ERR_ARG, "warps per block %lld (0..8)", v);
        h->warps = (int)v;
        return h->field_set ? check_shape(h, "aniso3_set_option") : ANISO_OK;
    case ANISO_OPT_SEGMENT:
        if (v < 0 || v > 64) return fail(ANISO_ERR_ARG, "segment %lld (0..64)", v);
        h->seg = (int)v;
        return h->field_set ? check_shape(h, "aniso3_set_option") : ANISO_OK;
    case ANISO_OPT_FIELD_FP16:
        if (h->field_set && (v != 0) != (h->field_fp16 != 0))
            return fail(ANISO_ERR_STATE, "field storage is fixed once the field is set");
        h->field_fp16 = v != 0;
        return ANISO_OK;
    case ANISO_OPT_KAHAN:
    case ANISO_OPT_ORDER:
    case ANISO_OPT_GRAPH:
    case ANISO_OPT_PROFILE:
    case ANISO_OPT_FAST_PATH:
        if (v == 0) return ANISO_OK;  // the default: nothing to change
        return fail(ANISO_ERR_UNSUPPORTED, "aniso3_set_option: option %d is two-dimensional only", key);
    default:
        return fail(ANISO_ERR_ARG, "aniso3_set_option: unknown key %d", key);
    }
}

extern "C" int aniso3_set_field(aniso3_t h, const void *bx, const void *by, const void *bz)
{
    if (!h) return fail(ANISO_ERR_ARG, "aniso3_set_field: null handle");
    if (!bx || !by || !bz) return fail(ANISO_ERR_ARG, "aniso3_set_field: null field pointer");
    if (h->field_fp16 && h->prec != PREC_FP32)
        return fail(ANISO_ERR_ARG, "aniso3_set_field: FP16 field storage needs FP32 precision");
    int rc = check_shape(h, "aniso3_set_field");
    if (rc) return rc;
    if (!h->field_set) {
        const size_t bytes = h->cells() * h->esz();
        for (auto &p : h->c) CU(cudaMalloc(&p, h->cells() * h->csz()));
        CU(cudaMalloc(&h->s1, bytes));
        CU(cudaMalloc(&h->s2, bytes));
        CU(cudaMalloc(&h->partials, 4 * TOTALS_BLOCKS * sizeof(double)));
        CU(cudaMalloc(&h->result, 4 * sizeof(double)));
        CU(cudaMalloc(&h->err, sizeof(unsigned)));
        CU(cudaMemsetAsync(h->err, 0, sizeof(unsigned), h->stream));
    }
    CU(launch_face_coeffs3(h->prec, h->field_fp16, bx, by, bz, h->n[0], h->n[1], h->n[2], h->bc,
                           h->chi_perp / h->chi_par, h->c, h->stream));
    h->field_set = true;
    return ANISO_OK;
}

// One update along axis d (0 x, 1 y, 2 z) of lines laid out for that axis:
// transverse axes a = d+1, b = d+2 (cyclic), line index kb * n[a] + ka.
static int enqueue3(aniso3_ctx *h, int d, const void *in, void *out, double lam, double mua, double mub,
                    bool transposed)
{
    const int a = (d + 1) % 3, b = (d + 2) % 3;
    Line2Args A{};
    A.jobs = nullptr;
    A.njobs = 1;
    A.limiter = h->limiter;
    A.err = h->err;
    Line2Job &J = A.one;
    J.Tin = in;
    J.Tout = out;
    J.g = h->c[3 * d];
    J.e = h->c[3 * d + 1];
    J.e2 = h->c[3 * d + 2];
    J.lam = lam;
    J.mu = mua;
    J.mu2 = mub;
    J.n = h->n[d];
    J.na = h->n[a];
    J.nlines = h->n[a] * h->n[b];
    J.per_line = J.per_cross = h->bc == ANISO_BC_PERIODIC ? 1 : 0;
    J.transpose_out = transposed ? 1 : 0;
    int nthreads;
    size_t smem;
    if (!line4_config(h->prec, J.n, transposed, h->warps, h->seg, &J.team, &J.lines_per_block, &nthreads, &smem))
        return fail(ANISO_ERR_UNSUPPORTED, "3-D line kernel cannot take n=%d", J.n);
    J.swz = line4_swizzle(h->prec, J.n, J.team);
    J.block0 = 0;
    J.nblocks = (J.nlines + J.lines_per_block - 1) / J.lines_per_block;
    CU(launch_line4_3d(h->prec, h->field_fp16, A, J.nblocks, nthreads, smem, h->stream));
    return ANISO_OK;
}

extern "C" int aniso3_step(aniso3_t h, void *T, double dt, int nsteps)
{
    if (!h) return fail(ANISO_ERR_ARG, "aniso3_step: null handle");
    if (!T) return fail(ANISO_ERR_ARG, "aniso3_step: T is NULL");
    if (!(dt > 0)) return fail(ANISO_ERR_ARG, "aniso3_step: dt must be > 0");
    if (nsteps < 0) return fail(ANISO_ERR_ARG, "aniso3_step: nsteps < 0");
    if (!h->field_set) return fail(ANISO_ERR_STATE, "aniso3_step: call aniso3_set_field first");
    if (((uintptr_t)T & 15) != 0) return fail(ANISO_ERR_ARG, "aniso3_step: T must be 16-byte aligned");
    const double c = h->chi_par * dt;
    double lam[3], mu[6];
    for (int d = 0; d < 3; ++d) {
        const int a = (d + 1) % 3, b = (d + 2) % 3;
        lam[d] = c / (h->d[d] * h->d[d]);
        mu[2 * d] = c / (h->d[d] * h->d[a]);
        mu[2 * d + 1] = c / (h->d[d] * h->d[b]);
    }
    int rc;
    for (int s = 0; s < nsteps; ++s) {
        if (h->scheme == ANISO_SCHEME_2STEP) {
            // T [z][y][x] -> s1 [x][z][y] -> s2 [y][x][z] -> T [z][y][x]
            if ((rc = enqueue3(h, 0, T, h->s1, lam[0], mu[0], mu[1], true))) return rc;
            if ((rc = enqueue3(h, 1, h->s1, h->s2, lam[1], mu[2], mu[3], true))) return rc;
            if ((rc = enqueue3(h, 2, h->s2, T, lam[2], mu[4], mu[5], true))) return rc;
        } else {
            // per axis: half-coefficient update with the transverse terms
            // (same layout), then a purely implicit half update (transposed)
            if ((rc = enqueue3(h, 0, T, h->s1, 0.5 * lam[0], mu[0], mu[1], false))) return rc;
            if ((rc = enqueue3(h, 0, h->s1, h->s2, 0.5 * lam[0], 0.0, 0.0, true))) return rc;
            if ((rc = enqueue3(h, 1, h->s2, h->s1, 0.5 * lam[1], mu[2], mu[3], false))) return rc;
            if ((rc = enqueue3(h, 1, h->s1, h->s2, 0.5 * lam[1], 0.0, 0.0, true))) return rc;
            if ((rc = enqueue3(h, 2, h->s2, h->s1, 0.5 * lam[2], mu[4], mu[5], false))) return rc;
            if ((rc = enqueue3(h, 2, h->s1, T, 0.5 * lam[2], 0.0, 0.0, true))) return rc;
        }
    }
    return ANISO_OK;
}

static int check_err3(aniso3_ctx *h)
{
    unsigned flag = 0;
    CU(cudaMemcpy(&flag, h->err, sizeof flag, cudaMemcpyDeviceToHost));
    if (flag) {
        CU(cudaMemset(h->err, 0, sizeof(unsigned)));
        return fail(ANISO_ERR_NONFINITE, "a 3-D step produced a non-finite temperature");
    }
    return ANISO_OK;
}

extern "C" int aniso3_total(aniso3_t h, const void *T, double *sum, double *tmin, double *tmax,
                            long long *nonfinite)
{
    if (!h) return fail(ANISO_ERR_ARG, "aniso3_total: null handle");
    if (!h->field_set) return fail(ANISO_ERR_STATE, "aniso3_total: call aniso3_set_field first");
    if (!T) return fail(ANISO_ERR_ARG, "aniso3_total: T is NULL");
    CU(launch_totals(h->prec, T, h->cells(), h->partials, h->result, h->stream));
    double r[4];
    CU(cudaMemcpyAsync(r, h->result, sizeof r, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (sum) *sum = r[0];
    if (tmin) *tmin = r[1];
    if (tmax) *tmax = r[2];
    if (nonfinite) *nonfinite = (long long)r[3];
    return check_err3(h);
}

extern "C" int aniso3_sync(aniso3_t h)
{
    if (!h) return fail(ANISO_ERR_ARG, "aniso3_sync: null handle");
    CU(cudaStreamSynchronize(h->stream));
    if (!h->err) return ANISO_OK;
    return check_err3(h);
}

extern "C" void aniso3_destroy(aniso3_t h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free3(h);
    delete h;
}
