// line2_kernel.cuh -- vectorised contiguous-line update (Eq. xup on rows; Eq.
// yup on a column-major copy), the fast path of the step.
//
// Same arithmetic as line_sweep_kernel (delta form, segment elimination,
// PCR of the segment-end unknowns; see sweep_kernels.cuh), reorganised so
// that every global and shared access moves 16 bytes:
//  - a line of n cells is m = n/V chunks of V = 16/sizeof(R) cells;
//    segments are whole chunks, so the segment walks read and write whole
//    16-byte chunks of shared memory;
//  - shared arrays are stored chunk-swizzled (chunk c at c ^ ((c>>3)&7)), so
//    the 8 lanes of a 16-byte shared-memory phase that walk 8 different
//    segments, and lanes that touch 8 consecutive chunks, hit 8 different
//    bank groups;
//  - the output is written either line-major or transposed (position-major,
//    `nlines` wide): the x-update writes T* column-major so that the
//    y-update reads its columns as contiguous lines and writes T^{n+1} back
//    row-major -- no separate transpose passes.
#pragma once
#include "sweep_kernels.cuh"

namespace aniso {

template <typename R> struct V16;
template <> struct V16<float> {
    typedef float4 T;
    enum { N = 4 };
    static __device__ __forceinline__ void unpack(const float4 &v, float *o)
    {
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
    static __device__ __forceinline__ float4 pack(const float *o) { return make_float4(o[0], o[1], o[2], o[3]); }
};
template <> struct V16<double> {
    typedef double2 T;
    enum { N = 2 };
    static __device__ __forceinline__ void unpack(const double2 &v, double *o)
    {
        o[0] = v.x;
        o[1] = v.y;
    }
    static __device__ __forceinline__ double2 pack(const double *o) { return make_double2(o[0], o[1]); }
};

// N coefficients of one chunk (16 bytes of T) as R.
__device__ __forceinline__ void ld_coef_chunk(const float *p, float *o)
{
    V16<float>::unpack(__ldg(reinterpret_cast<const float4 *>(p)), o);
}
__device__ __forceinline__ void ld_coef_chunk(const double *p, double *o)
{
    V16<double>::unpack(__ldg(reinterpret_cast<const double2 *>(p)), o);
}
__device__ __forceinline__ void ld_coef_chunk(const __half *p, float *o)
{
    const uint2 raw = __ldg(reinterpret_cast<const uint2 *>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&raw.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&raw.y));
    o[0] = a.x;
    o[1] = a.y;
    o[2] = b.x;
    o[3] = b.y;
}

// Chunk swizzle: within each complete group of 8 chunks, chunk c is stored at
// c ^ ((c >> 3) & 7); the incomplete tail group (chunks >= mfull) is stored
// unswizzled so that every index stays inside the line's m chunks.
// The same from shared memory (plain loads).
__device__ __forceinline__ void ld_coef_chunk_smem(const float *p, float *o)
{
    V16<float>::unpack(*reinterpret_cast<const float4 *>(p), o);
}
__device__ __forceinline__ void ld_coef_chunk_smem(const double *p, double *o)
{
    V16<double>::unpack(*reinterpret_cast<const double2 *>(p), o);
}
__device__ __forceinline__ void ld_coef_chunk_smem(const __half *p, float *o)
{
    const uint2 raw = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&raw.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&raw.y));
    o[0] = a.x;
    o[1] = a.y;
    o[2] = b.x;
    o[3] = b.y;
}

__device__ __forceinline__ int swz_chunk(int c, int mfull) { return c < mfull ? c ^ ((c >> 3) & 7) : c; }

// van Leer L(L(a,b),L(c,d)) in FP32 with one division.  With a,b the two
// differences of one cell and c,d those of the other, when all four share a
// strict sign the nesting equals 4pq / (p(c+d) + q(a+b)), p = ab, q = cd.
// Branch-free: p and q are clamped at 0 (a sign change within a cell gives
// 0), and a sign change between the cells, (a+b)(c+d) <= 0, gives 0; products
// below 1e-18 (differences below ~1e-9) also give 0, which keeps the
// denominator a normal number.
__device__ __forceinline__ float vanleer4_fast(float a, float b, float c, float d)
{
    const float p = a * b, q = c * d;
    const float sab = a + b, scd = c + d;
    const bool ok = (p > 1e-18f) & (q > 1e-18f) & (sab * scd > 0.f);
    const float den = fmaf(p, scd, q * sab);
    const float r = __fdividef(4.f * p * q, den);
    return ok ? r : 0.f;
}

template <typename R> __device__ __forceinline__ R limit4_v2(int lim, R a, R b, R c, R d)
{
    return limit4<R>(lim, a, b, c, d);
}
template <> __device__ __forceinline__ float limit4_v2<float>(int lim, float a, float b, float c, float d)
{
    if (lim == LIM_VANLEER) return vanleer4_fast(a, b, c, d);
    return limit4<float>(lim, a, b, c, d);
}

// K: compensated state (hi in Tin/Tout, lo in TinLo/ToutLo; line-major output
// only): differences are formed as (hi_a - hi_b) + (lo_a - lo_b), and each
// line's compensated sum of delta (zero in exact arithmetic) is removed before
// the double-word update hi + lo + delta.
template <typename R, typename C, bool K>
__global__ void __launch_bounds__(512, 2) line2_kernel(Line2Args args)
{
    typedef typename V16<R>::T VT;
    constexpr int N = V16<R>::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Line2Job J;
    if (threadIdx.x == 0)
        J = args.jobs ? args.jobs[args.block_job ? args.block_job[blockIdx.x] : find_job(args.jobs, args.njobs)]
                      : args.one;
    __syncthreads();

    const int lim = args.limiter;
    const int P = J.team, n = J.n, m = n / N, nl = J.nlines, LPB = J.lines_per_block;
    const int logP = __ffs(P) - 1;  // P is a power of two
    const int tm = threadIdx.x >> logP, t = threadIdx.x & (P - 1);
    const int line0 = (blockIdx.x - J.block0) * LPB;
    const int line = line0 + tm;
    const bool active = line < nl;
    const int lc = active ? line : nl - 1;
    int lu = lc + 1, ld = lc - 1;
    if (lu >= nl) lu = J.per_cross ? 0 : nl - 1;  // mirrored ghost line
    if (ld < 0) ld = J.per_cross ? nl - 1 : 0;
    const R *Tin = static_cast<const R *>(J.Tin);
    const R *rc = Tin + (size_t)lc * n, *ru = Tin + (size_t)lu * n, *rd = Tin + (size_t)ld * n;
    const R *TinL = static_cast<const R *>(J.TinLo);  // K only
    const R *rcl = K ? TinL + (size_t)lc * n : nullptr, *rul = K ? TinL + (size_t)lu * n : nullptr,
            *rdl = K ? TinL + (size_t)ld * n : nullptr;
    const C *G = static_cast<const C *>(J.g) + (size_t)lc * n;
    const C *E = static_cast<const C *>(J.e) + (size_t)lc * n;
    const R lam = (R)J.lam, mu = (R)J.mu;
    const bool per_line = J.per_line != 0;
    bool bad = false;  // a non-finite output of this thread

    const int LS = 3 * n + N;  // per-line stride (the extra chunk skews lines across banks)
    R *sF = reinterpret_cast<R *>(smem_raw) + tm * LS;  // F, then rho, then delta
    R *sG = sF + n;                                      // g, then alpha
    R *sQ = sG + n;                                      // gamma
    VT *vF = reinterpret_cast<VT *>(sF), *vG = reinterpret_cast<VT *>(sG), *vQ = reinterpret_cast<VT *>(sQ);
    const int mfull = m & ~7;
    auto swz = [mfull](int c) { return swz_chunk(c, mfull); };
    auto at = [&](int k) { return swz(k / N) * N + (k & (N - 1)); };
    const unsigned full = 0xffffffffu;

    // ---- A: face fluxes F_p (p+1/2) and normal coefficients, chunk by chunk
    {
        const int width = P < 32 ? P : 32;
        const int lane_in = t & (width - 1);
        const VT *vd = reinterpret_cast<const VT *>(rd), *vc = reinterpret_cast<const VT *>(rc),
                 *vu = reinterpret_cast<const VT *>(ru);
        const VT *wd = reinterpret_cast<const VT *>(rdl), *wc = reinterpret_cast<const VT *>(rcl),
                 *wu = reinterpret_cast<const VT *>(rul);
        for (int c0 = 0; c0 < m; c0 += P) {
            const int c = c0 + t;
            const int cl = c < m ? c : m - 1;
            R Td[N], Tc[N], Tu[N], Gv[N], Ev[N];
            R Ld[N] = {}, Lc[N] = {}, Lu[N] = {};  // low parts (K only)
            V16<R>::unpack(vd[cl], Td);
            V16<R>::unpack(vc[cl], Tc);
            V16<R>::unpack(vu[cl], Tu);
            if (K) {
                V16<R>::unpack(wd[cl], Ld);
                V16<R>::unpack(wc[cl], Lc);
                V16<R>::unpack(wu[cl], Lu);
            }
            ld_coef_chunk(G + cl * N, Gv);
            ld_coef_chunk(E + cl * N, Ev);
            R nd = __shfl_down_sync(full, Td[0], 1, width);
            R nc = __shfl_down_sync(full, Tc[0], 1, width);
            R nu = __shfl_down_sync(full, Tu[0], 1, width);
            R ndl = R(0), ncl = R(0), nul = R(0);
            if (K) {
                ndl = __shfl_down_sync(full, Ld[0], 1, width);
                ncl = __shfl_down_sync(full, Lc[0], 1, width);
                nul = __shfl_down_sync(full, Lu[0], 1, width);
            }
            if (c < m) {
                if (lane_in == width - 1 || c + 1 >= m) {
                    int p1 = (c + 1) * N;
                    if (p1 >= n) p1 = per_line ? 0 : n - 1;
                    nd = rd[p1];
                    nc = rc[p1];
                    nu = ru[p1];
                    if (K) {
                        ndl = rdl[p1];
                        ncl = rcl[p1];
                        nul = rul[p1];
                    }
                }
                R Fo[N];
#pragma unroll
                for (int v = 0; v < N; ++v) {
                    const R d1 = v + 1 < N ? Td[v + 1] : nd, d1l = v + 1 < N ? Ld[v + 1] : ndl;
                    const R c1 = v + 1 < N ? Tc[v + 1] : nc, c1l = v + 1 < N ? Lc[v + 1] : ncl;
                    const R u1 = v + 1 < N ? Tu[v + 1] : nu, u1l = v + 1 < N ? Lu[v + 1] : nul;
                    const R dT = limit4_v2<R>(lim, dif<R, K>(u1, u1l, c1, c1l), dif<R, K>(c1, c1l, d1, d1l),
                                              dif<R, K>(Tu[v], Lu[v], Tc[v], Lc[v]),
                                              dif<R, K>(Tc[v], Lc[v], Td[v], Ld[v]));
                    Fo[v] = lam * Gv[v] * dif<R, K>(c1, c1l, Tc[v], Lc[v]) + mu * Ev[v] * dT;
                }
                vF[swz(c)] = V16<R>::pack(Fo);
                vG[swz(c)] = V16<R>::pack(Gv);
            }
        }
    }
    __syncthreads();

    // ---- B1: segment = chunks [c_lo, c_hi), cells [s, e]; bottom-up elimination
    const int c_lo = (t * m) >> logP, c_hi = ((t + 1) * m) >> logP;
    const int s = c_lo * N;
    {
        const int sm1 = s == 0 ? n - 1 : s - 1;
        const R Fsm1 = sF[at(sm1)], gsm1 = sG[at(sm1)];
        if (P > 32) __syncthreads();
        else __syncwarp();
        // (the previous segment overwrites its chunks below; its last cell was read above)
        R rho1 = R(0), alp1 = R(0), gam1 = R(-1);
        R qp = R(0), qq = R(1), qw = R(0);
        R ae, be, ce, re;
        R f[N] = {}, gg[N] = {}, fp[N] = {}, gp[N] = {};
        auto load_prev = [&](int cc) {
            if (cc > c_lo) {
                V16<R>::unpack(vF[swz(cc - 1)], fp);
                V16<R>::unpack(vG[swz(cc - 1)], gp);
            } else {
                fp[N - 1] = Fsm1;
                gp[N - 1] = gsm1;
            }
        };
        auto eliminate = [&](int v, R Fkm, R gkm, R *ro, R *ao, R *go) {
            const R a = -lam * gkm, c = -lam * gg[v];
            const R b = R(1) - a - c;
            const R inv = Num<R>::div(R(1), b - c * alp1);
            const R alp = a * inv, gam = -c * gam1 * inv, rho = (f[v] - Fkm - c * rho1) * inv;
            ro[v] = rho;
            ao[v] = alp;
            go[v] = gam;
            qp = qp + qq * rho;
            qw = qw - qq * gam;
            qq = -qq * alp;
            rho1 = rho;
            alp1 = alp;
            gam1 = gam;
        };
        // last chunk: its last cell is row e (the bottom equation), the rest eliminate
        int cc = c_hi - 1;
        V16<R>::unpack(vF[swz(cc)], f);
        V16<R>::unpack(vG[swz(cc)], gg);
        load_prev(cc);
        {
            R ro[N], ao[N], go[N];
            ae = -lam * gg[N - 2 >= 0 ? N - 2 : 0];
            ce = -lam * gg[N - 1];
            be = R(1) - ae - ce;
            re = f[N - 1] - f[N - 2];
            ro[N - 1] = ao[N - 1] = go[N - 1] = R(0);
#pragma unroll
            for (int v = N - 2; v >= 0; --v) eliminate(v, v > 0 ? f[v - 1] : fp[N - 1], v > 0 ? gg[v - 1] : gp[N - 1], ro, ao, go);
            vF[swz(cc)] = V16<R>::pack(ro);
            vG[swz(cc)] = V16<R>::pack(ao);
            vQ[swz(cc)] = V16<R>::pack(go);
        }
        for (--cc; cc >= c_lo; --cc) {
#pragma unroll
            for (int v = 0; v < N; ++v) {
                f[v] = fp[v];
                gg[v] = gp[v];
            }
            load_prev(cc);
            R ro[N], ao[N], go[N];
#pragma unroll
            for (int v = N - 1; v >= 0; --v) eliminate(v, v > 0 ? f[v - 1] : fp[N - 1], v > 0 ? gg[v - 1] : gp[N - 1], ro, ao, go);
            vF[swz(cc)] = V16<R>::pack(ro);
            vG[swz(cc)] = V16<R>::pack(ao);
            vQ[swz(cc)] = V16<R>::pack(go);
        }

        // ---- R: reduced system of the line in the segment-end unknowns
        R X, Xm;
        if (P <= 32) {
            const int tn = (t + 1) & (P - 1);
            R rho_n = __shfl_sync(full, rho1, tn, P), alp_n = __shfl_sync(full, alp1, tn, P),
              gam_n = __shfl_sync(full, gam1, tn, P);
            X = pcr_warp<R>(make_reduced<R>(ae, be, ce, re, qp, qq, qw, rho_n, alp_n, gam_n), t, P);
            Xm = __shfl_sync(full, X, (t - 1) & (P - 1), P);
        } else {
            R *small = reinterpret_cast<R *>(smem_raw) + LPB * LS + tm * 8 * P;
            small[t] = rho1;
            small[P + t] = alp1;
            small[2 * P + t] = gam1;
            __syncthreads();
            const int tn = (t + 1) & (P - 1);
            Reduced<R> q = make_reduced<R>(ae, be, ce, re, qp, qq, qw, small[tn], small[P + tn],
                                           small[2 * P + tn]);
            __syncthreads();
            X = pcr_smem<R>(q, t, P, small, small + P, small + 2 * P, small + 3 * P, 1);
            small[4 * P + t] = X;
            __syncthreads();
            Xm = small[4 * P + ((t - 1) & (P - 1))];
        }

        // ---- B2: forward recovery, chunk by chunk (delta overwrites rho)
        R dprev = Xm;
        for (int c2 = c_lo; c2 < c_hi - 1; ++c2) {
            R ro[N], ao[N], go[N], d[N];
            V16<R>::unpack(vF[swz(c2)], ro);
            V16<R>::unpack(vG[swz(c2)], ao);
            V16<R>::unpack(vQ[swz(c2)], go);
#pragma unroll
            for (int v = 0; v < N; ++v) {
                d[v] = ro[v] - ao[v] * dprev - go[v] * X;
                dprev = d[v];
            }
            vF[swz(c2)] = V16<R>::pack(d);
        }
        {
            const int c2 = c_hi - 1;
            R ro[N], ao[N], go[N], d[N];
            V16<R>::unpack(vF[swz(c2)], ro);
            V16<R>::unpack(vG[swz(c2)], ao);
            V16<R>::unpack(vQ[swz(c2)], go);
#pragma unroll
            for (int v = 0; v < N - 1; ++v) {
                d[v] = ro[v] - ao[v] * dprev - go[v] * X;
                dprev = d[v];
            }
            d[N - 1] = X;
            vF[swz(c2)] = V16<R>::pack(d);
        }
    }
    __syncthreads();

    // ---- C: T_new = T_old + delta
    if (K) {
        // compensated state (line-major output): remove the line's residual
        // sum of delta, then the double-word update of (hi, lo)
        CSum<R> acc;
        for (int c = t; c < m; c += P) {
            R d[N];
            V16<R>::unpack(vF[swz(c)], d);
#pragma unroll
            for (int v = 0; v < N; ++v) acc.add(d[v]);
        }
        double part = (double)acc.s + (double)acc.c;
        double lsum;
        if (P <= 32) {
            for (int o = 1; o < P; o <<= 1) part += __shfl_xor_sync(full, part, o, P);
            lsum = part;
        } else {
            // the PCR area of this line (8P words, 8-byte aligned), free since B2
            double *red = reinterpret_cast<double *>(reinterpret_cast<R *>(smem_raw) + LPB * LS + tm * 8 * P);
            red[t] = part;
            __syncthreads();
            if (t == 0) {
                double a = 0.0;
                for (int k = 0; k < P; ++k) a += red[k];
                red[P] = a;
            }
            __syncthreads();
            lsum = red[P];
        }
        R ch, cl;
        split_f64(lsum / (double)n, ch, cl);
        if (active) {
            const VT *vo = reinterpret_cast<const VT *>(rc), *wo = reinterpret_cast<const VT *>(rcl);
            VT *out = reinterpret_cast<VT *>(static_cast<R *>(J.Tout) + (size_t)lc * n);
            VT *outl = reinterpret_cast<VT *>(static_cast<R *>(J.ToutLo) + (size_t)lc * n);
            for (int c = t; c < m; c += P) {
                R to[N], tw[N], d[N], oh[N], ol[N];
                V16<R>::unpack(vo[c], to);
                V16<R>::unpack(wo[c], tw);
                V16<R>::unpack(vF[swz(c)], d);
                R sum = R(0);
#pragma unroll
                for (int v = 0; v < N; ++v) {
                    dw_update(to[v], tw[v], d[v], ch, cl, oh[v], ol[v]);
                    sum += oh[v];
                }
                bad |= !(fabs(sum) < R(INFINITY));
                out[c] = V16<R>::pack(oh);
                outl[c] = V16<R>::pack(ol);
            }
        }
    } else if (!J.transpose_out) {
        if (active) {
            const VT *vo = reinterpret_cast<const VT *>(rc);
            VT *out = reinterpret_cast<VT *>(static_cast<R *>(J.Tout) + (size_t)lc * n);
            for (int c = t; c < m; c += P) {
                R to[N], d[N];
                V16<R>::unpack(vo[c], to);
                V16<R>::unpack(vF[swz(c)], d);
                R sum = R(0);
#pragma unroll
                for (int v = 0; v < N; ++v) {
                    to[v] += d[v];
                    sum += to[v];
                }
                bad |= !(fabs(sum) < R(INFINITY));  // a NaN or infinity in the chunk
                out[c] = V16<R>::pack(to);
            }
        }
    } else {
        // out[p][line] (position-major, nl wide): thread (group q4 of N lines,
        // position p), group fastest, reads the N deltas of position p (one
        // scalar per line, consecutive positions across lanes: no bank
        // conflicts) and T_old, and writes the N lines as one 16-byte store.
        R *out = static_cast<R *>(J.Tout);
        const int quads = LPB / N;  // a power of two in this mode
        const int logQ = __ffs(quads) - 1;
        const int q4 = threadIdx.x & (quads - 1);
        const int l0 = q4 * N;
        const R *src[N];
        const R *sl[N];
#pragma unroll
        for (int v = 0; v < N; ++v) {
            const int ln = line0 + l0 + v < nl ? line0 + l0 + v : nl - 1;
            src[v] = Tin + (size_t)ln * n;
            sl[v] = reinterpret_cast<R *>(smem_raw) + (l0 + v) * LS;
        }
        const bool vec_ok = (nl & (N - 1)) == 0 && line0 + l0 + N <= nl;
        const int pstride = blockDim.x >> logQ;
        for (int p = threadIdx.x >> logQ; p < n; p += pstride) {
            const int ap = at(p);
            R o[N];
            R sum = R(0);
#pragma unroll
            for (int v = 0; v < N; ++v) {
                o[v] = src[v][p] + sl[v][ap];
                sum += o[v];
            }
            bad |= !(fabs(sum) < R(INFINITY));
            R *dst = out + (size_t)p * nl + line0 + l0;
            if (vec_ok) {
                *reinterpret_cast<VT *>(dst) = V16<R>::pack(o);
            } else {
#pragma unroll
                for (int v = 0; v < N; ++v)
                    if (line0 + l0 + v < nl) dst[v] = o[v];
            }
        }
    }
    if (bad) atomicOr(args.err, 1u);
}

}  // namespace aniso
