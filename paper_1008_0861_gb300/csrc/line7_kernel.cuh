// line7_kernel.cuh -- lines cut across the blocks of a thread-block cluster
// (FP32; n = CS * np cells, np = 1024 or 2048, CS = 1, 2, 4 or 8 blocks).
//
// Same update as the other line kernels (Eq. xup on rows, Eq. yup on the
// column-major T*; delta form, bottom-up segment elimination, reduced system
// of the segment-end unknowns, recovery, transposed store).  A line of 16384
// cells needs 192 KB of line state, so one block could hold only one line and
// could not write its output transposed in vectors.  Here block r of a
// cluster holds cells [r np, (r+1) np) of four lines (12 B a cell of line
// state), and each line's piece belongs to a team of 64 lanes (two warps,
// 32 cells a lane at np = 2048).
//
// The reduced system of a line (one unknown X_t per lane, 64 CS of them) is
// solved in two levels:
//  - within each warp, the 31 unknowns of lanes 0..30 are expressed through
//    the two interface unknowns around them, b_{g-1} (lane 31 of the warp
//    before, in this block or the previous one) and b_g (lane 31 of this
//    warp):  X_t = p_t + q_t b_{g-1} + w_t b_g, by PCR over the warp's lanes
//    with three right-hand sides (warp shuffles, no barrier);
//  - lane 31's own equation, with those expressions substituted, couples
//    b_{g-1}, b_g and b_{g+1}: a cyclic tridiagonal system of G = 2 CS
//    interface unknowns per line.  Every warp publishes the 16 numbers that
//    system needs in its block's shared memory; after one cluster barrier one
//    warp per line in every block reads all G warps' numbers through
//    distributed shared memory and solves the system by PCR over G lanes, so
//    every block holds the same b.
// Both levels are Schur complements of the line's M-matrix, so they stay
// diagonally dominant M-matrices and the PCR steps divide by nonzero pivots.
//
// The face before a piece (its first row's lower face) is computed by the
// piece's lane 0 from global memory with the same operations, rounded the same
// way, as the previous piece computes it as its last face.
//
// K: compensated state (hi + lo FP32 pairs).  Differences are formed as
// (hi_a - hi_b) + (lo_a - lo_b); in exact arithmetic the sum of delta over a
// whole line is zero (the right-hand side telescopes and every column of the
// line matrix sums to one), so the line's compensated sum of the computed
// delta is rounding residual: every block adds the per-block partials of the
// line (one more cluster barrier, read in rank order, so every block gets the
// same sum) and removes it evenly while T_new = T_old + delta is formed in
// double-word arithmetic.
//
// Cluster barriers are hardware barriers (barrier.cluster arrive / wait),
// reached by every thread of every block of the cluster in the same order:
// there is no early return.  A block's shared memory must stay valid while
// others read it, so every block waits on the cluster once more before it
// exits.
#pragma once
#include "line4_kernel.cuh"

namespace aniso {

__device__ __forceinline__ unsigned cl_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cl_size()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cl_id()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
// Arrival that orders nothing: it only says this block has finished reading
// the others' shared memory (every value read has been used by then).
__device__ __forceinline__ void cl_arrive_relaxed()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
// Shared-window address of the same variable in block `rank` of the cluster.
__device__ __forceinline__ unsigned cl_map(const void *p, unsigned rank)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ float4 cl_ld4(unsigned addr)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}
__device__ __forceinline__ float2 cl_ld2(unsigned addr)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}
// Double-word FP32 sum (ah + al) + (bh + bl), renormalised.
__device__ __forceinline__ void dw_add(float ah, float al, float bh, float bl, float &sh, float &sl)
{
    float t, e;
    two_sum(ah, bh, t, e);
    e += al + bl;
    fast_two_sum(t, e, sh, sl);
}

// Face flux of the delta form at the face between cells a and a + 1:
// lg (T_{a+1} - T_a) + (mu e) L(v_a, v_{a+1}), rounded in a fixed order so
// that two blocks computing the same face agree bit for bit.
template <bool VL>
__device__ __forceinline__ float flux7(int lim, float lg, float mue, float dT, float va, float vb)
{
    return __fmaf_rn(lg, dT, __fmul_rn(mue, level<float, VL>(lim, va, vb)));
}
template <bool K> __device__ __forceinline__ float dif7(float ah, float al, float bh, float bl)
{
    return K ? __fadd_rn(__fsub_rn(ah, bh), __fsub_rn(al, bl)) : __fsub_rn(ah, bh);
}

constexpr int L7_P = 64;     // lanes of a line's team in a block
constexpr int L7_WPL = 2;    // warps of a team
constexpr int L7_LPB = 4;    // lines a block holds
constexpr int L7_THREADS = L7_P * L7_LPB;
constexpr int L7_PUB = 16;   // numbers a warp publishes for the interface system

// TM: each lane's gamma goes to its own tensor-memory lane instead of shared
// memory, so a block holds two arrays of its lines' state in shared memory and
// three blocks fit an SM.  TO: each lane's chunks of T_old (hi and lo with K)
// wait in its TMEM lane from the flux phase to phase C instead of being read
// again (TM implies it).
template <typename C, bool VL, bool K, bool TM, bool TO = TM>
__global__ void __launch_bounds__(L7_THREADS, TM ? 3 : 2) line7_kernel(Line2Args args)
{
    typedef float R;
    typedef float4 VT;
    constexpr int N = 4, P = L7_P, WPL = L7_WPL, LPB = L7_LPB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) float s_pub[LPB][WPL][L7_PUB];  // per warp: the interface system's inputs
    __shared__ float s_b[LPB][32];             // interface unknowns b_g of each line
    __shared__ float s_ex[LPB][2][P];          // lane t's last face (F, lam g) for lane t + 1
    __shared__ float s_fb[LPB][2];             // the face before the piece (F, lam g)
    __shared__ float s_wpart[LPB][WPL][2];      // K: per warp, sum of delta (double-word)
    __shared__ __align__(8) float s_lpart[LPB][2];  // K: per line, this block's part
    __shared__ float s_corr[LPB][2];            // K: per line, the line's sum / n

    const Line2Job &J = args.one;
    const int lim = args.limiter;
    const int CS = (int)cl_size(), rk = (int)cl_rank();
    const int n = J.n, np = n / CS, m = np / N, nl = J.nlines;
    const int G = WPL * CS;  // interface unknowns of a line
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lb = warp / WPL, wl = warp - lb * WPL;
    const int t = wl * 32 + lane;  // lane within the line's team
    const int line0 = (int)cl_id() * LPB;
    const int line = line0 + lb;
    const bool active = line < nl;
    const int lc = active ? line : nl - 1;
    int lu = lc + 1, ld = lc - 1;
    if (lu >= nl) lu = J.per_cross ? 0 : nl - 1;  // mirrored ghost line
    if (ld < 0) ld = J.per_cross ? nl - 1 : 0;
    const size_t p0 = (size_t)rk * np;  // first cell of the piece
    const size_t q0 = p0 / N;            // its first 4-cell quad
    // Input layout: separate hi / lo arrays (n floats a line), or (ilv) one
    // array of quads, 4 hi then 4 lo values per 4 cells (2 n floats a line).
    const bool ilv_in = K && J.ilv_in, ilv_out = K && J.ilv_out;
    const size_t ls = ilv_in ? 2 * (size_t)n : (size_t)n;
    auto vi = [ilv_in](size_t qc) { return ilv_in ? 2 * qc : qc; };                    // 16-byte index of quad qc
    auto si = [ilv_in](size_t q) { return ilv_in ? (((q >> 2) << 3) | (q & 3)) : q; };  // index of cell q
    const R *Tin = static_cast<const R *>(J.Tin);
    const R *Lc = Tin + (size_t)lc * ls, *Lu = Tin + (size_t)lu * ls, *Ld = Tin + (size_t)ld * ls;
    const R *TinL = ilv_in ? Tin + N : static_cast<const R *>(J.TinLo);
    const R *Lcl = K ? TinL + (size_t)lc * ls : nullptr, *Lul = K ? TinL + (size_t)lu * ls : nullptr,
            *Ldl = K ? TinL + (size_t)ld * ls : nullptr;
    const C *Gl = static_cast<const C *>(J.g) + (size_t)lc * n;
    const C *El = static_cast<const C *>(J.e) + (size_t)lc * n;
    const R lam = (R)J.lam, mu = (R)J.mu;
    const unsigned full = 0xffffffffu;

    const int U = m / P;  // chunks of a lane's segment (m is a multiple of P)
    const int c_lo = t * U;
    const int V = U;      // chunk rounds of the coalesced phases
    const int mfull = m & ~7, logU = 31 - __clz(U);
    constexpr int NARR = TM ? 2 : 3;                                     // shared arrays a line
    VT *sA = reinterpret_cast<VT *>(smem_raw) + (size_t)lb * NARR * m;  // F -> rho -> delta -> T_new (hi)
    VT *sB = sA + m;                                                     // lam*g -> alpha -> (K) T_new lo
    VT *sC = sA + 2 * m;                                                 // gamma (shared-memory form)
    // TMEM forms: warp 0 allocates the block's 128 columns now; the address
    // is read after the barrier that follows the first loads.  Warp w: lanes
    // 32 (w % 4) .. + 31, columns 64 (w / 4) .. + 63: with TM gamma of the
    // lane's segment chunk u at 4 u and its chunk of T_old of round v (from the
    // flux phase, for phase C, which takes the same chunks) at 32 + 4 v; with
    // TO alone (the compensated state) T_old's hi at 4 v and lo at 32 + 4 v.
    static_assert(!TM || TO, "the tensor-memory form keeps T_old there too");
    static_assert(!(TM && K), "the compensated state keeps gamma in shared memory");
    constexpr unsigned TM7_COLS = 128;
    constexpr unsigned COL_T = TM ? 32u : 0u, COL_TLO = 32u;
    __shared__ unsigned s_tmem;
    unsigned tm_lane = 0;
    if (TO) {
        if (warp == 0) tm_alloc(&s_tmem, TM7_COLS);
        tm_fence_before();
    }
    auto swz = [mfull, logU](int c) { return c < mfull ? c ^ ((c >> logU) & 7) : c; };

    // The block's rows of this piece into L2 (a hint): input lines line0 - 1
    // .. line0 + 4 (clamped) and the four lines' coefficients.
    if (threadIdx.x < 6) {
        const int l = max(0, min(line0 - 1 + (int)threadIdx.x, nl - 1));
        if (ilv_in) {
            l2_prefetch(Tin + (size_t)l * ls + 2 * p0, 2 * (size_t)np * sizeof(R));
        } else {
            l2_prefetch(Tin + (size_t)l * n + p0, (size_t)np * sizeof(R));
            if (K) l2_prefetch(static_cast<const R *>(J.TinLo) + (size_t)l * n + p0, (size_t)np * sizeof(R));
        }
    } else if (threadIdx.x < 6 + LPB) {
        const int l = min(line0 + (int)threadIdx.x - 6, nl - 1);
        l2_prefetch(static_cast<const C *>(J.g) + (size_t)l * n + p0, (size_t)np * sizeof(C));
        l2_prefetch(static_cast<const C *>(J.e) + (size_t)l * n + p0, (size_t)np * sizeof(C));
    }

    // ---- A: face fluxes and lam*g of the piece, coalesced (lane t: chunks
    // v*P + t), last round first with the next loads in flight.  The cell
    // after a chunk comes from the next lane by a shuffle; the warp's last
    // lane and the piece's last chunk read it directly.
    {
        const VT *vc = reinterpret_cast<const VT *>(Lc), *vd = reinterpret_cast<const VT *>(Ld),
                 *vu = reinterpret_cast<const VT *>(Lu);
        const VT *vcl = K ? reinterpret_cast<const VT *>(Lcl) : nullptr,
                 *vdl = K ? reinterpret_cast<const VT *>(Ldl) : nullptr,
                 *vul = K ? reinterpret_cast<const VT *>(Lul) : nullptr;
        typedef decltype(ld_raw(Gl)) CT;
        struct In {
            VT c, d, u;
            VT cl, dl, ul;  // K only
            CT g, e;
            R nc, nd, nu, ncl, ndl, nul;  // the cell after the chunk, where needed
        };
        auto load = [&](int v) {
            In x;
            const int c = v * P + t;
            const size_t vq = vi(q0 + c);
            x.c = vc[vq];
            x.d = vd[vq];
            x.u = vu[vq];
            if (K) {
                x.cl = vcl[vq];
                x.dl = vdl[vq];
                x.ul = vul[vq];
            }
            x.g = ld_raw(Gl + p0 + (size_t)c * N);
            x.e = ld_raw(El + p0 + (size_t)c * N);
            x.nc = x.nd = x.nu = x.ncl = x.ndl = x.nul = R(0);
            if (lane == 31 || c == m - 1) {
                size_t q = p0 + (size_t)N * (c + 1);
                if (q >= (size_t)n) q = J.per_line ? 0 : n - 1;
                q = si(q);
                x.nc = Lc[q];
                x.nd = Ld[q];
                x.nu = Lu[q];
                if (K) {
                    x.ncl = Lcl[q];
                    x.ndl = Ldl[q];
                    x.nul = Lul[q];
                }
            }
            return x;
        };
        auto body = [&](const In &x, int v) {
            const int c = v * P + t;
            R Tc[N], Td[N], Tu[N], Tcl[N], Tdl[N], Tul[N], Gv[N], Ev[N];
            V16<R>::unpack(x.c, Tc);
            V16<R>::unpack(x.d, Td);
            V16<R>::unpack(x.u, Tu);
            if (K) {
                V16<R>::unpack(x.cl, Tcl);
                V16<R>::unpack(x.dl, Tdl);
                V16<R>::unpack(x.ul, Tul);
            } else {
#pragma unroll
                for (int j = 0; j < N; ++j) Tcl[j] = Tdl[j] = Tul[j] = R(0);
            }
            if (TO) {  // warp-wide
                tm_st4(tm_lane + COL_T + 4u * (unsigned)v, Tc[0], Tc[1], Tc[2], Tc[3]);
                if (K) tm_st4(tm_lane + COL_TLO + 4u * (unsigned)v, Tcl[0], Tcl[1], Tcl[2], Tcl[3]);
            }
            unpack_raw(x.g, Gv);
            unpack_raw(x.e, Ev);
            R vv[N];
#pragma unroll
            for (int j = 0; j < N; ++j)
                vv[j] = level<R, VL>(lim, dif7<K>(Tu[j], Tul[j], Tc[j], Tcl[j]), dif7<K>(Tc[j], Tcl[j], Td[j], Tdl[j]));
            R nT = __shfl_down_sync(full, Tc[0], 1), nTl = K ? __shfl_down_sync(full, Tcl[0], 1) : R(0);
            R nv = __shfl_down_sync(full, vv[0], 1);
            if (lane == 31 || c == m - 1) {
                nT = x.nc;
                nTl = x.ncl;
                nv = level<R, VL>(lim, dif7<K>(x.nu, x.nul, x.nc, x.ncl), dif7<K>(x.nc, x.ncl, x.nd, x.ndl));
            }
            R F[N], lg[N];
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const R Tnx = j + 1 < N ? Tc[j + 1] : nT, Tnxl = j + 1 < N ? Tcl[j + 1] : nTl;
                const R vnx = j + 1 < N ? vv[j + 1] : nv;
                lg[j] = __fmul_rn(lam, Gv[j]);
                F[j] = flux7<VL>(lim, lg[j], __fmul_rn(mu, Ev[j]), dif7<K>(Tnx, Tnxl, Tc[j], Tcl[j]), vv[j], vnx);
            }
            sA[swz(c)] = V16<R>::pack(F);
            sB[swz(c)] = V16<R>::pack(lg);
        };
        if (K) {  // one round ahead (twice the loads a round)
            In cur = load(V - 1);
            if (TO) {  // the block's TMEM address, the first loads in flight
                __syncthreads();
                tm_fence_after();
                tm_lane = s_tmem + ((unsigned)(32 * (warp & 3)) << 16) + 64u * (unsigned)(warp >> 2);
            }
            for (int v = V - 1; v >= 0; --v) {
                const In x = cur;
                if (v >= 1) cur = load(v - 1);
                body(x, v);
            }
        } else {  // two rounds ahead
            In cur = load(V - 1);
            In nxt = V >= 2 ? load(V - 2) : cur;
            if (TO) {  // the block's TMEM address, the first loads in flight
                __syncthreads();
                tm_fence_after();
                tm_lane = s_tmem + ((unsigned)(32 * (warp & 3)) << 16) + 64u * (unsigned)(warp >> 2);
            }
            for (int v = V - 1; v >= 0; --v) {
                const In x = cur;
                cur = nxt;
                if (v >= 2) nxt = load(v - 2);
                body(x, v);
            }
        }
        // the face before the piece: cells q = p0 - 1 (wrapping) and p0
        if (t == 0) {
            const size_t q = p0 > 0 ? p0 - 1 : (size_t)n - 1;
            R g1[1], e1[1];
            g1[0] = (R)Gl[q];
            e1[0] = (R)El[q];
            const size_t a0 = si(q), a1 = si(p0);
            const R c0 = Lc[a0], d0 = Ld[a0], u0 = Lu[a0], c1 = Lc[a1], d1 = Ld[a1], u1 = Lu[a1];
            const R c0l = K ? Lcl[a0] : R(0), d0l = K ? Ldl[a0] : R(0), u0l = K ? Lul[a0] : R(0);
            const R c1l = K ? Lcl[a1] : R(0), d1l = K ? Ldl[a1] : R(0), u1l = K ? Lul[a1] : R(0);
            const R va = level<R, VL>(lim, dif7<K>(u0, u0l, c0, c0l), dif7<K>(c0, c0l, d0, d0l));
            const R vb = level<R, VL>(lim, dif7<K>(u1, u1l, c1, c1l), dif7<K>(c1, c1l, d1, d1l));
            const R lgq = __fmul_rn(lam, g1[0]);
            s_fb[lb][0] = flux7<VL>(lim, lgq, __fmul_rn(mu, e1[0]), dif7<K>(c1, c1l, c0, c0l), va, vb);
            s_fb[lb][1] = lgq;
        }
    }
    // T_old's tensor-memory stores complete before phase C reads them back
    // (the TM form's elimination waits again after its gamma stores)
    if (TO) tm_wait_st();
    __syncthreads();

    // ---- B1: bottom-up elimination of lane t's segment (as line6)
    R rho1 = R(0), alp1 = R(0), gam1 = R(-1);
    R qp = R(0), qq = R(1), qw = R(0);
    R ae = R(0), be = R(1), ce = R(0), re = R(0);
    R Fpend = R(0), lgpend = R(0), Flast = R(0), lglast = R(0);
    R ro[N], ao[N], go[N];
    auto elim = [&](R Fk, R Fkm, R lgk, R lgkm, R &ro_, R &ao_, R &go_) {
        // row k: -lgkm d_{k-1} + (1 + lgkm + lgk) d_k - lgk d_{k+1} = Fk - Fkm
        const R inv = Fast<R>::rcp((R(1) + lgkm + lgk) + lgk * alp1);
        const R alp = -lgkm * inv, gam = lgk * gam1 * inv, rho = ((Fk - Fkm) + lgk * rho1) * inv;
        ro_ = rho;
        ao_ = alp;
        go_ = gam;
        qp = qp + qq * rho;
        qw = qw - qq * gam;
        qq = -qq * alp;
        rho1 = rho;
        alp1 = alp;
        gam1 = gam;
    };
    {
#pragma unroll
        for (int v = 0; v < N; ++v) ro[v] = ao[v] = go[v] = R(0);
        for (int u = U - 1; u >= 0; --u) {
            const int c = c_lo + u;
            R F[N], lg[N], co[N], cao[N], cgo[N];
            V16<R>::unpack(sA[swz(c)], F);
            V16<R>::unpack(sB[swz(c)], lg);
            if (u == U - 1) {
                ae = -lg[N - 2];
                ce = -lg[N - 1];
                be = R(1) - ae - ce;
                re = F[N - 1] - F[N - 2];
                Flast = F[N - 1];
                lglast = lg[N - 1];
                co[N - 1] = cao[N - 1] = cgo[N - 1] = R(0);
#pragma unroll
                for (int j = N - 2; j >= 1; --j) elim(F[j], F[j - 1], lg[j], lg[j - 1], co[j], cao[j], cgo[j]);
            } else {
                elim(Fpend, F[N - 1], lgpend, lg[N - 1], ro[0], ao[0], go[0]);
                sA[swz(c + 1)] = V16<R>::pack(ro);
                sB[swz(c + 1)] = V16<R>::pack(ao);
                if (TM) tm_st4(tm_lane + 4u * (unsigned)(u + 1), go[0], go[1], go[2], go[3]);  // warp-wide
                else sC[swz(c + 1)] = V16<R>::pack(go);
#pragma unroll
                for (int j = N - 1; j >= 1; --j) elim(F[j], F[j - 1], lg[j], lg[j - 1], co[j], cao[j], cgo[j]);
            }
            Fpend = F[0];
            lgpend = lg[0];
#pragma unroll
            for (int j = 1; j < N; ++j) {
                ro[j] = co[j];
                ao[j] = cao[j];
                go[j] = cgo[j];
            }
        }
    }
    s_ex[lb][0][t] = Flast;
    s_ex[lb][1][t] = lglast;
    __syncthreads();
    {
        const R Fb = t > 0 ? s_ex[lb][0][t - 1] : s_fb[lb][0];
        const R lgb = t > 0 ? s_ex[lb][1][t - 1] : s_fb[lb][1];
        elim(Fpend, Fb, lgpend, lgb, ro[0], ao[0], go[0]);
        sA[swz(c_lo)] = V16<R>::pack(ro);
        sB[swz(c_lo)] = V16<R>::pack(ao);
        if (TM) {
            tm_st4(tm_lane, go[0], go[1], go[2], go[3]);
            tm_wait_st();  // the recovery reads these columns back
        } else {
            sC[swz(c_lo)] = V16<R>::pack(go);
        }
    }

    // Phase C's first two chunks of T_old start loading now.
    const VT *vcC = reinterpret_cast<const VT *>(Lc);
    const VT *vcCl = K ? reinterpret_cast<const VT *>(Lcl) : nullptr;
    VT pre0{}, pre1{};  // (TMEM forms: T_old waits in tensor memory)
    VT pre0l = make_float4(0.f, 0.f, 0.f, 0.f), pre1l = pre0l;
    if (!TO) {
        pre0 = vcC[vi(q0 + t)];
        pre1 = V >= 2 ? vcC[vi(q0 + t + P)] : pre0;
        if (K) {
            pre0l = vcCl[vi(q0 + t)];
            pre1l = V >= 2 ? vcCl[vi(q0 + t + P)] : pre0l;
        }
    }

    // ---- R1: the warp's unknowns through the interface unknowns around it
    R pX, qX, wX;
    {
        const R rho_n = __shfl_down_sync(full, rho1, 1), alp_n = __shfl_down_sync(full, alp1, 1),
                gam_n = __shfl_down_sync(full, gam1, 1);
        Reduced<R> q = make_reduced<R>(ae, be, ce, re, qp, qq, qw, rho_n, alp_n, gam_n);
        R Q = R(0), W = R(0);
        if (lane == 0) {  // coupling to b_{g-1} moves to the right-hand side
            Q = -q.L;
            q.L = R(0);
        }
        if (lane == 30) {  // coupling to b_g
            W = -q.U;
            q.U = R(0);
        }
        if (lane == 31) {  // b_g itself: an identity row here
            q.L = R(0);
            q.D = R(1);
            q.U = R(0);
            q.Rr = R(0);
        }
        for (int h = 1; h < 32; h <<= 1) {
            const int tm = (lane - h) & 31, tp = (lane + h) & 31;
            const R Lm = __shfl_sync(full, q.L, tm), Dm = __shfl_sync(full, q.D, tm);
            const R Um = __shfl_sync(full, q.U, tm), Rm = __shfl_sync(full, q.Rr, tm);
            const R Qm = __shfl_sync(full, Q, tm), Wm = __shfl_sync(full, W, tm);
            const R Lp = __shfl_sync(full, q.L, tp), Dp = __shfl_sync(full, q.D, tp);
            const R Up = __shfl_sync(full, q.U, tp), Rp = __shfl_sync(full, q.Rr, tp);
            const R Qp = __shfl_sync(full, Q, tp), Wp = __shfl_sync(full, W, tp);
            const R k1 = Fast<R>::div(q.L, Dm), k2 = Fast<R>::div(q.U, Dp);
            q.D = q.D - k1 * Um - k2 * Lp;
            q.Rr = q.Rr - k1 * Rm - k2 * Rp;
            Q = Q - k1 * Qm - k2 * Qp;
            W = W - k1 * Wm - k2 * Wp;
            q.L = -k1 * Lm;
            q.U = -k2 * Up;
        }
        const R inv = Fast<R>::rcp(q.L + q.D + q.U);
        pX = q.Rr * inv;
        qX = Q * inv;
        wX = W * inv;
        float *pub = s_pub[lb][wl];
        if (lane == 0) {
            pub[0] = rho1;
            pub[1] = alp1;
            pub[2] = gam1;
            pub[3] = pX;
            pub[4] = qX;
            pub[5] = wX;
        } else if (lane == 30) {
            pub[6] = pX;
            pub[7] = qX;
            pub[8] = wX;
        } else if (lane == 31) {
            pub[9] = ae;
            pub[10] = be;
            pub[11] = ce;
            pub[12] = re;
            pub[13] = qp;
            pub[14] = qq;
            pub[15] = qw;
        }
    }
    cl_arrive();
    cl_wait();

    // ---- R2: the interface system of every line, solved in every block
    if (wl == 0) {
        const int g = lane & (G - 1);
        const unsigned base = cl_map(&s_pub[lb][g % WPL][0], (unsigned)(g / WPL));
        float v[L7_PUB];
#pragma unroll
        for (int k = 0; k < L7_PUB; k += 4) {
            const float4 w = cl_ld4(base + 4u * k);
            v[k] = w.x;
            v[k + 1] = w.y;
            v[k + 2] = w.z;
            v[k + 3] = w.w;
        }
        // the next warp's top map and its lane 0 in terms of (b_g, b_{g+1})
        const int gn = (g + 1) & (G - 1);
        const R rho_n = __shfl_sync(full, v[0], gn, G), alp_n = __shfl_sync(full, v[1], gn, G),
                gam_n = __shfl_sync(full, v[2], gn, G);
        const R p0n = __shfl_sync(full, v[3], gn, G), q0n = __shfl_sync(full, v[4], gn, G),
                w0n = __shfl_sync(full, v[5], gn, G);
        // lane 31's equation: L y30 + D b_g + U y32 = Rr
        const Reduced<R> e31 = make_reduced<R>(v[9], v[10], v[11], v[12], v[13], v[14], v[15], rho_n, alp_n, gam_n);
        Reduced<R> s;
        s.L = e31.L * v[7];
        s.D = e31.D + e31.L * v[8] + e31.U * q0n;
        s.U = e31.U * w0n;
        s.Rr = e31.Rr - e31.L * v[6] - e31.U * p0n;
        const R b = pcr_team<R>(s, g, G);
        if (lane < G) s_b[lb][lane] = b;
    }
    if (!K) cl_arrive_relaxed();  // this block reads no other block's memory after this
    __syncthreads();

    // ---- X_t and X_{t-1}
    R X, Xm;
    {
        const int gme = rk * WPL + wl;
        const R bm = s_b[lb][(gme - 1 + G) & (G - 1)], bme = s_b[lb][gme];
        X = lane == 31 ? bme : pX + qX * bm + wX * bme;
        Xm = __shfl_up_sync(full, X, 1);
        if (lane == 0) Xm = bm;
    }

    // ---- B2: forward recovery of lane t's segment (delta over rho)
    CSum<R> acc;
    {
        R dprev = Xm;
        for (int u = 0; u < U; ++u) {
            const int c = c_lo + u;
            R r4[N], a4[N], g4[N], d[N];
            V16<R>::unpack(sA[swz(c)], r4);
            V16<R>::unpack(sB[swz(c)], a4);
            if (TM) tm_ld4(tm_lane + 4u * (unsigned)u, g4);  // warp-wide
            else V16<R>::unpack(sC[swz(c)], g4);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                d[j] = (u == U - 1 && j == N - 1) ? X : r4[j] - a4[j] * dprev - g4[j] * X;
                dprev = d[j];
                if (K) acc.add(d[j]);
            }
            sA[swz(c)] = V16<R>::pack(d);
        }
    }

    // K: the line's compensated sum of delta, the same in every block
    R ch = R(0), clo = R(0);
    if (K) {
        // double-word FP32 throughout: lanes by a butterfly (both orders of
        // an exact two-sum give the same pair), warps and blocks in order
        float sh, sl;
        two_sum(acc.s, acc.c, sh, sl);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const float oh = __shfl_xor_sync(full, sh, o), ol = __shfl_xor_sync(full, sl, o);
            dw_add(sh, sl, oh, ol, sh, sl);
        }
        if (lane == 0) {
            s_wpart[lb][wl][0] = sh;
            s_wpart[lb][wl][1] = sl;
        }
        __syncthreads();
        if (threadIdx.x < LPB) {
            float ah = s_wpart[threadIdx.x][0][0], al = s_wpart[threadIdx.x][0][1];
#pragma unroll
            for (int w = 1; w < WPL; ++w) dw_add(ah, al, s_wpart[threadIdx.x][w][0], s_wpart[threadIdx.x][w][1], ah, al);
            s_lpart[threadIdx.x][0] = ah;
            s_lpart[threadIdx.x][1] = al;
        }
        cl_arrive();
        cl_wait();
        if (threadIdx.x < LPB) {
            float ah = R(0), al = R(0);
            for (int k = 0; k < CS; ++k) {
                const float2 b2 = cl_ld2(cl_map(&s_lpart[threadIdx.x][0], (unsigned)k));
                dw_add(ah, al, b2.x, b2.y, ah, al);
            }
            const float inv = 1.0f / (float)n;  // n is a power of two: exact, and so are the products
            s_corr[threadIdx.x][0] = ah * inv;
            s_corr[threadIdx.x][1] = al * inv;
        }
        cl_arrive_relaxed();
        __syncthreads();
        ch = s_corr[lb][0];
        clo = s_corr[lb][1];
    } else {
        __syncthreads();
    }

    // ---- C: T_new = T_old + delta, coalesced; staged for the store
    bool bad = false;
    for (int v = 0; v < V; ++v) {
        const int c = v * P + t;
        R to[N], tol[N], d[N];
        if (TO) {  // warp-wide
            tm_ld4(tm_lane + COL_T + 4u * (unsigned)v, to);
            if (K) tm_ld4(tm_lane + COL_TLO + 4u * (unsigned)v, tol);
        } else {
            V16<R>::unpack(pre0, to);
            if (K) V16<R>::unpack(pre0l, tol);
            pre0 = pre1;
            if (K) pre0l = pre1l;
            if (v + 2 < V) {
                pre1 = vcC[vi(q0 + c + 2 * P)];
                if (K) pre1l = vcCl[vi(q0 + c + 2 * P)];
            }
        }
        V16<R>::unpack(sA[swz(c)], d);
        R hi[N], lo[N];
        R sum = R(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            if (K) {
                dw_update(to[j], tol[j], d[j], ch, clo, hi[j], lo[j]);
            } else {
                hi[j] = to[j] + d[j];
                lo[j] = R(0);
            }
            sum += hi[j];
        }
        bad |= !(fabsf(sum) < INFINITY);
        if (!J.transpose_out) {
            if (active && ilv_out) {
                VT *o = reinterpret_cast<VT *>(static_cast<R *>(J.Tout) + (size_t)lc * 2 * n) + 2 * (q0 + c);
                o[0] = V16<R>::pack(hi);
                o[1] = V16<R>::pack(lo);
            } else if (active) {
                reinterpret_cast<VT *>(static_cast<R *>(J.Tout) + (size_t)lc * n + p0)[c] = V16<R>::pack(hi);
                if (K) reinterpret_cast<VT *>(static_cast<R *>(J.ToutLo) + (size_t)lc * n + p0)[c] = V16<R>::pack(lo);
            }
        } else {
            sA[swz(c)] = V16<R>::pack(hi);
            if (K) sB[swz(c)] = V16<R>::pack(lo);
        }
    }

    // ---- transposed store: out[p][line], the block's four lines in 16-byte
    // pieces; interleaved, each position's hi and lo pieces fill one 32-byte
    // sector (two neighbouring threads)
    if (J.transpose_out && ilv_out) {
        __syncthreads();
        R *out = static_cast<R *>(J.Tout);
        for (int idx = threadIdx.x; idx < 2 * np; idx += blockDim.x) {
            const int p = idx >> 1, half = idx & 1;
            const int sc = swz(p >> 2), j = p & 3;
            R o[N];
#pragma unroll
            for (int i = 0; i < N; ++i)
                o[i] = reinterpret_cast<const R *>(reinterpret_cast<const VT *>(smem_raw) + (size_t)i * NARR * m +
                                                   (size_t)half * m + sc)[j];
            *reinterpret_cast<VT *>(out + (size_t)(p0 + p) * 2 * nl + 2 * (size_t)line0 + N * half) = V16<R>::pack(o);
        }
    } else if (J.transpose_out) {
        __syncthreads();
        R *out = static_cast<R *>(J.Tout);
        R *outl = static_cast<R *>(J.ToutLo);
        const bool vec_ok = (nl & 3) == 0;
        for (int p = threadIdx.x; p < np; p += blockDim.x) {
            const int sc = swz(p >> 2), j = p & 3;
            R o[N], ol[N];
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const VT *base = reinterpret_cast<const VT *>(smem_raw) + (size_t)i * NARR * m;
                o[i] = reinterpret_cast<const R *>(base + sc)[j];
                if (K) ol[i] = reinterpret_cast<const R *>(base + m + sc)[j];
            }
            const size_t row = (size_t)(p0 + p) * nl + line0;
            if (vec_ok && line0 + N <= nl) {
                *reinterpret_cast<VT *>(out + row) = V16<R>::pack(o);
                if (K) *reinterpret_cast<VT *>(outl + row) = V16<R>::pack(ol);
            } else {
#pragma unroll
                for (int i = 0; i < N; ++i)
                    if (line0 + i < nl) {
                        out[row + i] = o[i];
                        if (K) outl[row + i] = ol[i];
                    }
            }
        }
    }
    if (bad && active) atomicOr(args.err, 1u);
    if (TO) {  // every warp is done with TMEM before the block frees it
        tm_fence_before();
        __syncthreads();
        if (warp == 0) {
            tm_fence_after();
            tm_dealloc(s_tmem, TM7_COLS);
        }
    }
    cl_wait();  // no block leaves while another may still read its shared memory
}

}  // namespace aniso
