// lbgb_colloid.cu -- particle kernels: node map and remap (destroy / create),
// wetting virtual densities with the solid-node Shan-Chen force, Ladd link
// forces, pair forces (cell list) and the rotational leap-frog integrator.
//
// Per-particle lattice work runs one 16x8 thread block per particle over the
// box of lattice points around its sphere.  Geometry is evaluated in the
// compute type of the populations (FP32 for the FP32 / FP16 forms): FP64
// arithmetic on GB300 runs at a small fraction of the FP32 rate and costs a
// whole warp even in a divergent branch, so it is kept out of per-link code.
// Node membership |x - r_p|^2 < R^2 is nevertheless decided exactly: points
// whose FP32 distance is within a safe margin of the sphere are re-tested in
// FP64.  Each thread accumulates its share of a per-particle sum with a
// compensated (Neumaier) sum in the compute type; the thread partials are
// merged in FP64 in a fixed order (warp shuffles, then warps in order), so
// the per-particle totals are FP64 and independent of scheduling.
#include "lbgb_internal.cuh"

namespace lbgb {

constexpr int BXP = 16, BYP = 8, PB = BXP * BYP;  // particle block
constexpr double REMAP_PAD = 0.75;
constexpr unsigned REMAP_GROUPS = 1;  // blocks per particle in the remap kernels

// geometry of particle p in compute type C
template <typename C>
struct PGeo {
    int lo[3], ext[3];  // box of lattice points
    int ip[3];          // floor(r_p)
    C fr[3];            // r_p - floor(r_p)
    C v[3], w[3];       // v(t-1/2), omega(t-1/2)
    double R;
    C R2;
};

template <typename C>
__device__ __forceinline__ PGeo<C> pgeo(const Lattice& L, int p, double pad) {
    PGeo<C> g;
    g.R = L.rad[p];
    g.R2 = C(g.R) * C(g.R);
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (sizeof(C) == 8) {
            double r = L.pos[3 * p + d];
            g.lo[d] = (int)floor(r - g.R - pad);
            g.ext[d] = (int)ceil(r + g.R + pad) - g.lo[d] + 1;
            g.ip[d] = (int)floor(r);
            g.fr[d] = C(r - (double)g.ip[d]);
            g.v[d] = C(L.vel[3 * p + d]);
            g.w[d] = C(L.omg[3 * p + d]);
        } else {
            // box from the snapshot: r = ip + fr with fr in [0, 1) (the box only
            // has to cover the working shell, which it does with a wide margin)
            g.ip[d] = L.ipos[3 * p + d];
            g.fr[d] = C(L.fsnap[9 * p + d]);
            g.v[d] = C(L.fsnap[9 * p + 3 + d]);
            g.w[d] = C(L.fsnap[9 * p + 6 + d]);
            float Rp = float(g.R) + float(pad);
            g.lo[d] = g.ip[d] + (int)floorf(float(g.fr[d]) - Rp);
            g.ext[d] = g.ip[d] + (int)ceilf(float(g.fr[d]) + Rp) - g.lo[d] + 1;
        }
    }
    return g;
}

// exact membership |a - r_p|^2 < R^2 (FP64 without contraction, as a plain
// double evaluation would decide it)
__device__ __noinline__ bool inside_exact(const Lattice& L, int p, int a, int b, int c) {
    double dx = (double)a - L.pos[3 * p], dy = (double)b - L.pos[3 * p + 1], dz = (double)c - L.pos[3 * p + 2];
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    double R = L.rad[p];
    return d2 < __dmul_rn(R, R);
}

template <typename C>
__device__ __forceinline__ bool inside(const Lattice& L, int p, const PGeo<C>& g, const C (&d)[3], int a, int b,
                                       int c) {
    if (sizeof(C) == 8) return inside_exact(L, p, a, b, c);
    C d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    C gap = d2 - g.R2;
    if (gap > C(1e-2) || gap < C(-1e-2)) return gap < C(0);
    return inside_exact(L, p, a, b, c);
}

// |d| within [R + lo, R + hi) (in the compute type, with the margins chosen
// by the callers well beyond its rounding): the shell where a kernel can have
// work, so that the rest of the box is skipped without memory traffic
template <typename C>
__device__ __forceinline__ bool in_shell(const PGeo<C>& g, const C (&d)[3], float lo, float hi) {
    float d2 = float(d[0]) * float(d[0]) + float(d[1]) * float(d[1]) + float(d[2]) * float(d[2]);
    float a = float(g.R) + lo, b = float(g.R) + hi;
    return (a <= 0.f || d2 >= a * a) && d2 < b * b;
}

// Visit the box points of particle p; f(X, Y, Z, s, a, b, c, d) gets the
// wrapped site, its index, the unwrapped point and its offset from r_p.  A
// grid of (particles, groups) splits each box into interleaved groups of
// planes, so that more independent blocks hide the latency of the loads.
template <typename C, typename Fn>
__device__ __forceinline__ void for_box(const Lattice& L, const PGeo<C>& g, Fn&& fn) {
    // the planes of the box are shared among the gridDim.y blocks of a particle
    for (int zz = blockIdx.y; zz < g.ext[2]; zz += gridDim.y) {
        int c = g.lo[2] + zz;
        if (!L.per[2] && (c < 0 || c >= L.nz)) continue;
        int Z = c < 0 ? c + L.nz : (c >= L.nz ? c - L.nz : c);
        for (int yy = threadIdx.y; yy < g.ext[1]; yy += BYP) {
            int b = g.lo[1] + yy;
            int Y = b < 0 ? b + L.ny : (b >= L.ny ? b - L.ny : b);
            for (int xx = threadIdx.x; xx < g.ext[0]; xx += BXP) {
                int a = g.lo[0] + xx;
                int X = a < 0 ? a + L.nx : (a >= L.nx ? a - L.nx : a);
                long long s = (long long)X + (long long)L.nx * ((long long)Y + (long long)L.ny * Z);
                C d[3] = {C(a - g.ip[0]) - g.fr[0], C(b - g.ip[1]) - g.fr[1], C(c - g.ip[2]) - g.fr[2]};
                fn(X, Y, Z, s, a, b, c, d);
            }
        }
    }
}

// Visit the box points of particle p whose distance from the centre lies in
// [R + lo, R + hi) (the in_shell test, so the set is exactly that of a box
// scan), one (y, z) row of the box per thread: the x range of a row that can
// reach the shell is found from the row's distance to the centre (one or two
// intervals, widened by a point on each side), so a thin shell costs its own
// points instead of the whole box.  Sites are indexed in 32 bits.
template <typename C, typename Fn>
__device__ __forceinline__ void for_band(const Lattice& L, const PGeo<C>& g, float lo, float hi, Fn&& fn) {
    const int tid = threadIdx.y * BXP + threadIdx.x;
    const int nrow = g.ext[1] * g.ext[2];
    const float Rin = float(g.R) + lo, Rout = float(g.R) + hi;
    const float cxr = float(g.ip[0]) + float(g.fr[0]);  // x of the centre (box frame)
    for (int r = tid; r < nrow; r += PB) {
        const int b = g.lo[1] + r % g.ext[1], c = g.lo[2] + r / g.ext[1];
        if (!L.per[2] && (c < 0 || c >= L.nz)) continue;
        const C dy = C(b - g.ip[1]) - g.fr[1], dz = C(c - g.ip[2]) - g.fr[2];
        const float q = float(dy) * float(dy) + float(dz) * float(dz);
        const float ho = Rout * Rout - q;
        if (ho < -1.f) continue;
        const float xo = sqrtf(fmaxf(ho, 0.f)) + 1.f;
        const float hin = Rin > 0.f ? Rin * Rin - q : -1.f;
        const float xi = hin > 1.f ? sqrtf(hin) - 1.f : 0.f;  // |dx| >= xi can be in the shell
        const int Y = b < 0 ? b + L.ny : (b >= L.ny ? b - L.ny : b);
        const int Z = c < 0 ? c + L.nz : (c >= L.nz ? c - L.nz : c);
        const int row = L.nx * (Y + L.ny * Z);
        // x with |a - cx| in [xi, xo]: the left and right intervals (one if xi = 0)
        const int aL0 = (int)floorf(cxr - xo), aL1 = (int)ceilf(cxr - xi);
        const int aR0 = (int)floorf(cxr + xi), aR1 = (int)ceilf(cxr + xo);
        const int split = xi > 0.f && aL1 < aR0;
        for (int part = 0; part < 1 + split; part++) {
            const int a0 = part == 0 ? aL0 : aR0, a1 = (part == 0 && split) ? aL1 : aR1;
            for (int a = a0; a <= a1; a++) {
                const C dx = C(a - g.ip[0]) - g.fr[0];
                const C d[3] = {dx, dy, dz};
                if (!in_shell<C>(g, d, lo, hi)) continue;
                const int X = a < 0 ? a + L.nx : (a >= L.nx ? a - L.nx : a);
                fn(X, Y, Z, (long long)(row + X), a, b, c, d);
            }
        }
    }
}

// Visit the box points of particle p whose distance from the centre lies in
// [R + lo, R + hi), with the work packed onto consecutive threads (used by
// the kernels whose per-point work is heavy; the remap kernels, whose work is
// a few loads per point, scan the box directly): the box is
// scanned 128 points at a time, the points in the shell are appended to a
// shared list in box order (warp ballots, warps in order), and whenever 128
// are queued (and at the end) each thread takes one.  A thin shell fills
// about a sixth of the box, so without packing most lanes of a warp would
// idle through the per-point work.  The assignment of points to threads
// depends only on the geometry, so per-thread partial sums are reproducible.
template <typename C, typename Fn>
__device__ __forceinline__ void for_shell(const Lattice& L, const PGeo<C>& g, float lo, float hi, Fn&& fn) {
    __shared__ int list[2 * PB];
    __shared__ int wcnt[PB / 32];
    __shared__ int count;
    const int tid = threadIdx.y * BXP + threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ex = g.ext[0], exy = g.ext[0] * g.ext[1], total = exy * g.ext[2];
    auto decode = [&](int t, int& X, int& Y, int& Z, int& a, int& b, int& c, long long& s, C (&d)[3]) -> bool {
        a = g.lo[0] + t % ex;
        b = g.lo[1] + (t / ex) % g.ext[1];
        c = g.lo[2] + t / exy;
        if (!L.per[2] && (c < 0 || c >= L.nz)) return false;
        X = a < 0 ? a + L.nx : (a >= L.nx ? a - L.nx : a);
        Y = b < 0 ? b + L.ny : (b >= L.ny ? b - L.ny : b);
        Z = c < 0 ? c + L.nz : (c >= L.nz ? c - L.nz : c);
        s = (long long)X + (long long)L.nx * ((long long)Y + (long long)L.ny * Z);
        d[0] = C(a - g.ip[0]) - g.fr[0];
        d[1] = C(b - g.ip[1]) - g.fr[1];
        d[2] = C(c - g.ip[2]) - g.fr[2];
        return true;
    };
    if (tid == 0) count = 0;
    __syncthreads();
    for (int base = 0; base < total; base += PB) {
        int t = base + tid;
        bool act = false;
        if (t < total) {
            int X, Y, Z, a, b, c;
            long long s;
            C d[3];
            act = decode(t, X, Y, Z, a, b, c, s, d) && in_shell<C>(g, d, lo, hi);
        }
        unsigned bal = __ballot_sync(0xffffffffu, act);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        int off = count, tot = 0;
        for (int w = 0; w < PB / 32; w++) {
            if (w < warp) off += wcnt[w];
            tot += wcnt[w];
        }
        if (act) list[off + __popc(bal & ((1u << lane) - 1u))] = t;
        __syncthreads();
        if (tid == 0) count += tot;
        __syncthreads();
        bool last = base + PB >= total;
        while (count >= PB || (last && count > 0)) {
            int n = count < PB ? count : PB;
            if (tid < n) {
                int X, Y, Z, a, b, c;
                long long s;
                C d[3];
                decode(list[tid], X, Y, Z, a, b, c, s, d);
                fn(X, Y, Z, s, a, b, c, d);
            }
            __syncthreads();
            int rest = count - n;
            if (tid < rest) list[tid] = list[n + tid];
            __syncthreads();
            if (tid == 0) count = rest;
            __syncthreads();
        }
    }
}

template <typename C>
__device__ __forceinline__ void crs(const C (&a)[3], const C (&b)[3], C (&o)[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Deterministic block reduction of M per-thread compensated partials into
// FP64 totals (thread 0 receives them in out).  Within a warp the (s, c)
// pairs are merged in the compute type with the same compensated rule (a
// fixed butterfly); lane m < M of warp 0 then converts the warp partials of
// value m to FP64 and merges them in warp order, so the FP64 work is a few
// instructions per block rather than per thread.
template <int M, typename C>
__device__ void block_reduce(CSum<C> (&part)[M], double* out) {
    __shared__ C sh_s[PB / 32][M], sh_c[PB / 32][M];
    __shared__ double sh_out[M];
    int tid = threadIdx.y * BXP + threadIdx.x;
    int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int m = 0; m < M; m++) {
        CSum<C> acc = part[m];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            C os = __shfl_down_sync(0xffffffffu, acc.s, off);
            C oc = __shfl_down_sync(0xffffffffu, acc.c, off);
            if (lane < off) {
                acc.add(os);
                acc.c += oc;
            }
        }
        if (lane == 0) {
            sh_s[warp][m] = acc.s;
            sh_c[warp][m] = acc.c;
        }
    }
    __syncthreads();
    if (warp == 0 && lane < M) {
        NSum t = {0.0, 0.0};
        for (int w = 0; w < PB / 32; w++) {
            NSum o = {double(sh_s[w][lane]), double(sh_c[w][lane])};
            t.merge(o);
        }
        sh_out[lane] = t.value();
    }
    __syncthreads();
    if (tid == 0)
        for (int m = 0; m < M; m++) out[m] = sh_out[m];
}

template <typename C, int M>
__device__ __forceinline__ void zero(CSum<C> (&a)[M]) {
#pragma unroll
    for (int m = 0; m < M; m++) a[m].s = a[m].c = C(0);
}

template <int PREC>
__device__ __forceinline__ typename Prec<PREC>::C site_rho(const Lattice& L, long long s, int k) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    const S* f = (const S*)L.f_cur;
    C r = 0;
#pragma unroll
    for (int i = 0; i < Q; i++)
        r += ld_pop(f + pop_index(k * Q + i, s, L.pstride), pop_shift<S, C>(L, k, i));
    return r;
}

// -------------------------------------------------- FP32 snapshot
__global__ void k_snapshot(Lattice L) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L.nc) return;
    for (int d = 0; d < 3; d++) {
        double r = L.pos[3 * p + d];
        int ip = (int)floor(r);
        L.ipos[3 * p + d] = ip;
        L.fsnap[9 * p + d] = float(r - (double)ip);
        L.fsnap[9 * p + 3 + d] = float(L.vel[3 * p + d]);
        L.fsnap[9 * p + 6 + d] = float(L.omg[3 * p + d]);
    }
}

// ------------------------------------------------------ initial node map
// First map after particles are added: nodes are claimed without momentum
// bookkeeping (Sec. 2.4).
template <int PREC>
__global__ void __launch_bounds__(PB) k_map_initial(Lattice L, int first) {
    typedef typename Prec<PREC>::C C;
    int p = first + blockIdx.x;
    PGeo<C> g = pgeo<C>(L, p, 0.0);
    for_box<C>(L, g, [&](int, int, int, long long s, int a, int b, int c, const C (&d)[3]) {
        if (!inside<C>(L, p, g, d, a, b, c)) return;
        int old = atomicCAS(L.owner + s, -1, p);
        if (old != -1 && old != p) atomicOr(L.flags, FLAG_OVERLAP);
        L.mask[s] = 1;
    });
}

// ------------------------------------------------------------- remap
// The nodes the remap of a step changes are listed (nb_chg, up to
// NB_CHG_CAP): the refill, the commit and the link classes then visit only
// them.  When more change, the list is left incomplete and every kernel that
// uses it falls back to scanning the particles' shells.
__device__ __forceinline__ void list_changed(const Lattice& L, long long s) {
    const int q = atomicAdd(L.nb_chg, 1);
    if (q < NB_CHG_CAP) L.nb_chg[8 + q] = (int)s;
}

// x_s - r_p (minimum image) and the particle's v, omega, in the compute type:
// FP32 / FP16 from the snapshot (integer cell + offset), FP64 from the state
template <typename C>
__device__ __forceinline__ void particle_frame(const Lattice& L, int p, int x, int y, int z, C (&d)[3], C (&v)[3],
                                               C (&w)[3]) {
    const int xs[3] = {x, y, z}, Ls[3] = {L.nx, L.ny, L.nz};
#pragma unroll
    for (int c = 0; c < 3; c++) {
        int ip;
        C fr;
        if (sizeof(C) == 8) {
            const double r = L.pos[3 * p + c];
            ip = (int)floor(r);
            fr = C(r - (double)ip);
            v[c] = C(L.vel[3 * p + c]);
            w[c] = C(L.omg[3 * p + c]);
        } else {
            ip = L.ipos[3 * p + c];
            fr = C(L.fsnap[9 * p + c]);
            v[c] = C(L.fsnap[9 * p + 3 + c]);
            w[c] = C(L.fsnap[9 * p + 6 + c]);
        }
        int dd = xs[c] - ip;
        if (L.per[c]) {
            if (2 * dd > Ls[c]) dd -= Ls[c];
            else if (2 * dd < -Ls[c]) dd += Ls[c];
        }
        d[c] = C(dd) - fr;
    }
}

// The remap kernels work on the points within 0.65 of the surface (a node
// changes side only within the distance moved, below 1/2 per step); their
// box reaches 0.75 beyond the sphere.
// Classify the points around particle p at its new position r_p(t):
//   fluid node now inside -> destroy (Eq. 24): its momentum rho u goes to p
//   node of p now outside -> create (handled by k_remap_create)
template <int PREC>
__global__ void __launch_bounds__(PB) k_remap_classify(Lattice L) {
    typedef typename Prec<PREC>::C C;
    int p = blockIdx.x;
    PGeo<C> g = pgeo<C>(L, p, REMAP_PAD);
    CSum<C> acc[6];
    zero(acc);
    for_box<C>(L, g, [&](int, int, int, long long s, int a, int b, int c, const C (&d)[3]) {
        // a node changes side only within the distance moved (< 1/2, checked
        // by the integrator) of the sphere
        if (!in_shell<C>(g, d, -0.65f, 0.65f)) return;
        int o = L.owner[s];
        if (inside<C>(L, p, g, d, a, b, c)) {
            if (o == -1) {
                if (atomicCAS(L.evt + s, 0, 4 * (p + 1) + 1) != 0) {
                    atomicOr(L.flags, FLAG_OVERLAP);
                    return;
                }
                list_changed(L, s);
                C fv[2][Q], rho[2], j[2][3], u[3], om;
                load_site<PREC>(L, (const typename Prec<PREC>::S*)L.f_cur, s, fv, rho, j);
                mixture<C>(L, rho, j, u, om);
                C rt = rho[0] + rho[1];
                C mom[3] = {rt * u[0], rt * u[1], rt * u[2]}, tq[3];
                crs<C>(d, mom, tq);
#pragma unroll
                for (int m = 0; m < 3; m++) {
                    acc[m].add(mom[m]);
                    acc[3 + m].add(tq[m]);
                }
            } else if (o != p) {
                atomicOr(L.flags, FLAG_OVERLAP);
            }
        } else if (o == p) {
            L.evt[s] = 4 * (p + 1) + 2;
            list_changed(L, s);
        }
    });
    double out[6];
    block_reduce<6, C>(acc, out);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int m = 0; m < 3; m++) {
            acc_add(L, acc_slot(L, ACC_FD, p, m), out[m]);
            acc_add(L, acc_slot(L, ACC_TD, p, m), out[3 + m]);
        }
}

// Refill the nodes released by p (Eq. 25): f = f^eq(rhobar^k, u_w) with
// rhobar^k the w_i-weighted mean over neighbours that are fluid before and
// after the remap, u_w = v_p + omega_p x (r - r_p); p loses (rhobar) u_w.
template <int PREC>
__global__ void __launch_bounds__(PB) k_remap_create(Lattice L) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    if (*L.nb_chg <= NB_CHG_CAP) return;  // the list kernel does it
    int p = blockIdx.x;
    PGeo<C> g = pgeo<C>(L, p, REMAP_PAD);
    CSum<C> acc[6];
    zero(acc);
    const int code = 4 * (p + 1) + 2;
    for_band<C>(L, g, -0.65f, 0.65f, [&](int X, int Y, int Z, long long s, int, int, int, const C (&d)[3]) {
        if (!in_shell<C>(g, d, -0.65f, 0.65f)) return;
        if (L.evt[s] != code) return;
        SiteNbr n = site_nbr(L, X, Y, Z);
        C num[2] = {0, 0}, den = 0;
        for (int i = 1; i < Q; i++) {
            if (nbr_is_wall(n, i)) continue;
            long long m = nbr_index(L, n, i);
            if (L.owner[m] != -1 || L.evt[m] != 0) continue;
            C w = wgt<C>(i);
            num[0] += w * site_rho<PREC>(L, m, 0);
            num[1] += w * site_rho<PREC>(L, m, 1);
            den += w;
        }
        C rb[2];
        for (int k = 0; k < 2; k++) rb[k] = den > C(0) ? num[k] / den : C(L.P.rho0[k]);
        C wxd[3], uw[3];
        crs<C>(g.w, d, wxd);
        for (int m = 0; m < 3; m++) uw[m] = g.v[m] + wxd[m];
        C uu = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
        S* f = (S*)L.f_cur;
        for (int k = 0; k < 2; k++)
            for (int i = 0; i < Q; i++)
                st_pop(f + pop_index(k * Q + i, s, L.pstride), feq<C>(i, rb[k], uw[0], uw[1], uw[2], uu),
                       pop_shift<S, C>(L, k, i));
        C rt = rb[0] + rb[1];
        C mom[3] = {-rt * uw[0], -rt * uw[1], -rt * uw[2]}, tq[3];
        crs<C>(d, mom, tq);
#pragma unroll
        for (int m = 0; m < 3; m++) {
            acc[m].add(mom[m]);
            acc[3 + m].add(tq[m]);
        }
    });
    double out[6];
    block_reduce<6, C>(acc, out);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int m = 0; m < 3; m++) {
            acc_add(L, acc_slot(L, ACC_FC, p, m), out[m]);
            acc_add(L, acc_slot(L, ACC_TC, p, m), out[3 + m]);
        }
}

// Commit the new node map of particle p.
template <int PREC>
__global__ void __launch_bounds__(PB) k_remap_commit(Lattice L) {
    typedef typename Prec<PREC>::C C;
    if (*L.nb_chg <= NB_CHG_CAP) return;  // the list kernel does it
    int p = blockIdx.x;
    PGeo<C> g = pgeo<C>(L, p, REMAP_PAD);
    for_band<C>(L, g, -0.65f, 0.65f, [&](int, int, int, long long s, int, int, int, const C (&d)[3]) {
        if (!in_shell<C>(g, d, -0.65f, 0.65f)) return;
        int e = L.evt[s];
        if (e == 4 * (p + 1) + 1) {
            int old = atomicCAS(L.owner + s, -1, p);
            if (old != -1) atomicOr(L.flags, FLAG_OVERLAP);
            L.mask[s] = 1;
            L.evt[s] = 0;
        } else if (e == 4 * (p + 1) + 2) {
            L.owner[s] = -1;
            L.mask[s] = 0;
            L.evt[s] = 0;
        }
    });
}

// The refill (Eq. 25) of the listed nodes a particle released, one thread
// per listed node (k_remap_create's work when the list is complete): the
// momentum (rhobar) u_w each one carries off its particle is added to F_c,
// T_c as its own fixed-point term.
template <int PREC>
__global__ void k_remap_create_list(Lattice L) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    const int cnt = *L.nb_chg;
    if (cnt > NB_CHG_CAP) return;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const long long s = L.nb_chg[8 + t];
        const int code = L.evt[s];
        if ((code & 3) != 2) continue;
        const int p = code / 4 - 1;
        const long long xy = (long long)L.nx * L.ny;
        const int Z = (int)(s / xy), r = (int)(s - (long long)Z * xy), Y = r / L.nx, X = r - Y * L.nx;
        SiteNbr n = site_nbr(L, X, Y, Z);
        C num[2] = {0, 0}, den = 0;
        for (int i = 1; i < Q; i++) {
            if (nbr_is_wall(n, i)) continue;
            long long m = nbr_index(L, n, i);
            if (L.owner[m] != -1 || L.evt[m] != 0) continue;
            C w = wgt<C>(i);
            num[0] += w * site_rho<PREC>(L, m, 0);
            num[1] += w * site_rho<PREC>(L, m, 1);
            den += w;
        }
        C rb[2];
        for (int k = 0; k < 2; k++) rb[k] = den > C(0) ? num[k] / den : C(L.P.rho0[k]);
        C d[3], v[3], w[3], wxd[3], uw[3];
        particle_frame<C>(L, p, X, Y, Z, d, v, w);
        crs<C>(w, d, wxd);
        for (int m = 0; m < 3; m++) uw[m] = v[m] + wxd[m];
        C uu = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
        S* f = (S*)L.f_cur;
        for (int k = 0; k < 2; k++)
            for (int i = 0; i < Q; i++)
                st_pop(f + pop_index(k * Q + i, s, L.pstride), feq<C>(i, rb[k], uw[0], uw[1], uw[2], uu),
                       pop_shift<S, C>(L, k, i));
        C rt = rb[0] + rb[1];
        C mom[3] = {-rt * uw[0], -rt * uw[1], -rt * uw[2]}, tq[3];
        crs<C>(d, mom, tq);
        for (int m = 0; m < 3; m++) {
            acc_add(L, acc_slot(L, ACC_FC, p, m), mom[m]);
            acc_add(L, acc_slot(L, ACC_TC, p, m), tq[m]);
        }
    }
}

// Commit the listed nodes (k_remap_commit's work when the list is complete).
__global__ void k_remap_commit_list(Lattice L) {
    const int cnt = *L.nb_chg;
    if (cnt > NB_CHG_CAP) return;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const long long s = L.nb_chg[8 + t];
        const int e = L.evt[s], p = e / 4 - 1;
        if ((e & 3) == 1) {
            int old = atomicCAS(L.owner + s, -1, p);
            if (old != -1) atomicOr(L.flags, FLAG_OVERLAP);
            L.mask[s] = 1;
        } else if ((e & 3) == 2) {
            L.owner[s] = -1;
            L.mask[s] = 0;
        }
        L.evt[s] = 0;
    }
}

// The link-class word of site s = (x, y, z) from the node map (NB_*).
__device__ uint32_t link_classes(const Lattice& L, int x, int y, int z, long long s) {
    const SiteNbr n = site_nbr(L, x, y, z);
    const bool solid = L.mask[s] != 0;
    uint32_t bits = 0, multi = 0;
    int p0 = -1;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        if (nbr_is_wall(n, i)) continue;
        const long long m = nbr_index(L, n, i);
        const bool ms = L.mask[m] != 0;
        bits |= (uint32_t)(ms != solid) << i;
        if (!solid && ms) {
            const int p = L.owner[m];
            multi |= p0 >= 0 && p != p0 ? NB_MULTI : 0u;
            p0 = p0 < 0 ? p : p0;
        }
    }
    return bits | multi | (solid ? NB_SOLID : 0u);
}

// every site (grid: x chunks, y, z)
__global__ void k_link_classes_all(Lattice L) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= L.nx) return;
    const long long s = (long long)x + (long long)L.nx * ((long long)y + (long long)L.ny * z);
    L.nb[s] = link_classes(L, x, y, z, s);
}

// The sites within one link of the nodes the remap changed (the map is
// final): a site next to two changed nodes is rewritten with the same word
// by both.  When more nodes changed than the list holds, every site.
__global__ void k_link_classes_changed(Lattice L) {
    const int cnt = *L.nb_chg;
    const long long nt = (long long)gridDim.x * blockDim.x;
    long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cnt > NB_CHG_CAP) {
        for (long long s = t0; s < L.N; s += nt) {
            const long long xy = (long long)L.nx * L.ny;
            const int z = (int)(s / xy), r = (int)(s - (long long)z * xy), y = r / L.nx, x = r - y * L.nx;
            L.nb[s] = link_classes(L, x, y, z, s);
        }
        return;
    }
    for (long long t = t0; t < (long long)cnt * Q; t += nt) {
        const long long c = L.nb_chg[8 + t / Q];
        const int i = (int)(t % Q);
        const long long xy = (long long)L.nx * L.ny;
        const int z = (int)(c / xy), r = (int)(c - (long long)z * xy), y = r / L.nx, x = r - y * L.nx;
        const SiteNbr n = site_nbr(L, x, y, z);
        if (i > 0 && nbr_is_wall(n, i)) continue;
        int X = x, Y = y, Z = z;
        if (i > 0) {
            X = rc(0, i) > 0 ? n.xp : (rc(0, i) < 0 ? n.xm : x);
            Y = rc(1, i) > 0 ? n.yp : (rc(1, i) < 0 ? n.ym : y);
            Z = rc(2, i) > 0 ? n.zp : (rc(2, i) < 0 ? n.zm : z);
        }
        const long long s = (long long)X + (long long)L.nx * ((long long)Y + (long long)L.ny * Z);
        L.nb[s] = link_classes(L, X, Y, Z, s);
    }
}

// ------------------------------------------------------------ wetting
// Indices of the 18 neighbours of a site (-1 beyond a wall) and the bit set
// of those that are particle nodes; the 18 mask loads are independent, so
// they are in flight together.
__device__ __forceinline__ uint32_t nbr_solid(const Lattice& L, const SiteNbr& n, int (&m)[Q]) {
    uint32_t bits = 0;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        bool wall = nbr_is_wall(n, i);
        m[i] = wall ? -1 : (int)nbr_index(L, n, i);
        uint8_t v = wall ? 0 : __ldg(L.mask + m[i]);
        bits |= (uint32_t)(v != 0) << i;
    }
    return bits;
}

// Eq. 20 on every frontier node s (a particle node with at least one fluid
// neighbour): psi^k(s) = (1 + zeta^k) sum w_i rho^k / sum w_i over the fluid
// neighbours (with the Janus switch s of the node: 1 + s zeta^A, 1 - s zeta^B)
// neighbours, and Eq. 21 (repulsive sign):
// F_s = -G sum_k psi^k(s) sum w_i rho^kbar(s + c_i) c_i, added with its torque
// (x_s - r_p) x F_s to the fixed-point sums F_s, T_s of the owning particle
// (the step zeroes them in launch_remap).  A block loads psi^k and the owner
// map of a 32 x 8 tile (+ one-site ring) for all planes of its z chunk (+ one
// on each side) into shared memory in one batch, 12 bytes per site in
// coalesced rows; the frontier nodes of the chunk (from the link classes)
// are then packed onto consecutive threads, so that the per-node work runs
// with all lanes busy, and each takes its fluid neighbours from shared
// memory.  The densities rho^k of the fluid nodes are those of the full
// density pass of this step (k_density).
constexpr int VTX = 32, VTY = 8, VZC = 8;  // tile and planes per block

template <int PREC>
__global__ void __launch_bounds__(VTX* VTY) k_virtual(Lattice L, int store_terms, int zc) {
    typedef typename Prec<PREC>::C C;
    constexpr int NT = VTX * VTY, NPL = VZC + 2;
    extern __shared__ __align__(16) unsigned char vsm[];
    // planes z0-1 .. z0+zc of the tile + ring: node codes, then psi^A, psi^B
    int (*snd)[VTY + 2][VTX + 2] = reinterpret_cast<int (*)[VTY + 2][VTX + 2]>(vsm);
    // (psi^A, psi^B) pairs after the node codes (whose size is a multiple of 16 bytes)
    C (*sp)[VTY + 2][VTX + 2][2] =
        reinterpret_cast<C (*)[VTY + 2][VTX + 2][2]>(vsm + sizeof(int) * NPL * (VTY + 2) * (VTX + 2));
    __shared__ int cand[NT * VZC];
    __shared__ int wcnt[NT / 32];

    const int x0 = blockIdx.x * VTX, y0 = blockIdx.y * VTY;
    const int W = min(VTX, L.nx - x0), H = min(VTY, L.ny - y0);
    const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, L.nz), nz_b = z1 - z0;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * VTX + tx, lane = tid & 31, warp = tid >> 5;
    const bool act = tx < W && ty < H;
    const long long nxy = (long long)L.nx * L.ny;
    C* psi = (C*)L.psi;
    auto wrap_xy = [&](int lx, int ly) {
        int X = x0 + lx, Y = y0 + ly;
        X = X < 0 ? X + L.nx : (X >= L.nx ? X - L.nx : X);
        Y = Y < 0 ? Y + L.ny : (Y >= L.ny ? Y - L.ny : Y);
        return X + L.nx * Y;
    };
    const int own_xy = wrap_xy(tx, ty);
    const bool has_ring = tid < 2 * (W + 2) + 2 * H;
    int rlx, rly;
    if (tid < W + 2) { rlx = tid - 1; rly = -1; }
    else if (tid < 2 * (W + 2)) { rlx = tid - (W + 2) - 1; rly = H; }
    else if (tid < 2 * (W + 2) + H) { rlx = -1; rly = tid - 2 * (W + 2); }
    else { rlx = W; rly = tid - 2 * (W + 2) - H; }
    const int ring_xy = has_ring ? wrap_xy(rlx, rly) : 0;
    // every plane of the chunk at once (asynchronous copies, all in flight
    // together); a plane beyond a wall has no fluid node
    for (int q = 0; q < nz_b + 2; q++) {
        const int p = z0 - 1 + q;
        const bool wall = (p < 0 || p >= L.nz) && !L.per[2];
        const int Z = p < 0 ? p + L.nz : (p >= L.nz ? p - L.nz : p);
        const long long zoff = nxy * Z;
        auto put = [&](int ly, int lx, long long g) {
            if (wall) {
                snd[q][ly][lx] = ND_WALL;
                sp[q][ly][lx][0] = sp[q][ly][lx][1] = C(0);
                return;
            }
            cp_async_4(&snd[q][ly][lx], L.owner + g);
            if (sizeof(C) == 8) {
                cp_async_16(&sp[q][ly][lx][0], psi + 2 * g);
            } else {
                cp_async_8(&sp[q][ly][lx][0], psi + 2 * g);
            }
        };
        if (act) put(ty + 1, tx + 1, zoff + own_xy);
        if (has_ring) put(rly + 1, rlx + 1, zoff + ring_xy);
    }
    // the frontier nodes of the tile's own column (a particle node with a
    // fluid neighbour: its link classes), one bit per plane of the chunk
    unsigned front = 0;
    if (act)
        for (int q = 1; q <= nz_b; q++) {
            const uint32_t c = L.nb[nxy * (z0 + q - 1) + own_xy];
            front |= (unsigned)((c & NB_SOLID) && (c & NB_LINKS)) << q;
        }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    // the frontier nodes of the chunk, packed onto consecutive threads (in
    // plane, warp and lane order: fixed by the geometry)
    const int mine = __popc(front);
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wcnt[warp] = incl;
    __syncthreads();
    int off = incl - mine, tot = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; w++) {
        off += w < warp ? wcnt[w] : 0;
        tot += wcnt[w];
    }
    for (int q = 1; q <= nz_b; q++)
        if ((front >> q) & 1u) cand[off++] = q * NT + tid;
    __syncthreads();
    const C G = prm<C>(L.P.G, L.PF.G), zA = C(1) + C(L.P.zeta[0]), zB = C(1) + C(L.P.zeta[1]);
    // whole warps step through the list together (lanes past its end carry
    // no term), so that a warp whose nodes all belong to one particle adds
    // its terms with one set of atomics: the fixed-point words are summed
    // across the warp first (exact integer sums, so the bits do not depend
    // on the grouping)
    for (int base = warp * 32; base < tot; base += NT) {
        const int k = base + lane;
        bool has = false;
        int p = -1;
        C fs[3] = {0, 0, 0}, tq[3] = {0, 0, 0};
        if (k < tot) {
            const int e = cand[k], q = e / NT, t = e - q * NT, cx0 = t % VTX, cy0 = t / VTX;
            p = snd[q][cy0 + 1][cx0 + 1];
            C num[2] = {0, 0}, den = 0;
            C sA[3] = {0, 0, 0}, sB[3] = {0, 0, 0};
#pragma unroll
            for (int i = 1; i < Q; i++) {
                const int a = q + cz(i), yy = cy0 + 1 + cy(i), xx = cx0 + 1 + cx(i);
                const bool fl = snd[a][yy][xx] == ND_FLUID;
                C ra = fl ? sp[a][yy][xx][0] : C(0), rb = fl ? sp[a][yy][xx][1] : C(0);
                C w = fl ? wgt<C>(i) : C(0);
                num[0] += w * ra;
                num[1] += w * rb;
                den += w;
                sA[0] += w * ra * C(cx(i)); sA[1] += w * ra * C(cy(i)); sA[2] += w * ra * C(cz(i));
                sB[0] += w * rb * C(cx(i)); sB[1] += w * rb * C(cy(i)); sB[2] += w * rb * C(cz(i));
            }
            if (den > C(0)) {
                const int z = z0 + q - 1;
                const long long s = nxy * z + (x0 + cx0) + (long long)L.nx * (y0 + cy0);
                C d[3];
                // x_s - r_p (minimum image) from the integer cell and offset of r_p
                const int xs[3] = {x0 + cx0, y0 + cy0, z}, Ls[3] = {L.nx, L.ny, L.nz};
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    int ip;
                    C fr;
                    if (sizeof(C) == 8) {
                        double r = L.pos[3 * p + c];
                        ip = (int)floor(r);
                        fr = C(r - (double)ip);
                    } else {
                        ip = L.ipos[3 * p + c];
                        fr = C(L.fsnap[9 * p + c]);
                    }
                    int dd = xs[c] - ip;
                    if (L.per[c]) {
                        if (2 * dd > Ls[c]) dd -= Ls[c];
                        else if (2 * dd < -Ls[c]) dd += Ls[c];
                    }
                    d[c] = C(dd) - fr;
                }
                C fa = zA, fb = zB;
                if (L.P.janus) {
                    const C sw = janus_switch<C>(L, p, d);
                    fa = C(1) + sw * C(L.P.zeta[0]);
                    fb = C(1) - sw * C(L.P.zeta[1]);
                }
                const C pa = fa * num[0] / den;
                const C pb = fb * num[1] / den;
                psi[2 * s] = pa;
                psi[2 * s + 1] = pb;
                if (store_terms) {
#pragma unroll
                    for (int c = 0; c < 3; c++) fs[c] = -G * pa * sB[c] + -G * pb * sA[c];
                    crs<C>(d, fs, tq);
                    has = true;
                }
            }
        }
        if (!store_terms) continue;  // uniform across the block
        const unsigned any = __ballot_sync(0xffffffffu, has);
        if (!any) continue;
        const int p0 = __shfl_sync(0xffffffffu, p, __ffs(any) - 1);
        const bool one = __all_sync(0xffffffffu, !has || p == p0);
#pragma unroll
        for (int m = 0; m < 6; m++) {
            const C v = m < 3 ? fs[m] : tq[m - 3];
            unsigned long long w[2] = {0ull, 0ull};
            if (has && !acc_words(L, v, w)) w[0] = w[1] = 0ull;
            if (!one) {
                if (has) acc_add_words(L, acc_slot(L, m < 3 ? ACC_FS : ACC_TS, p, m % 3), w);
                continue;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                w[0] += __shfl_xor_sync(0xffffffffu, w[0], o);
                w[1] += __shfl_xor_sync(0xffffffffu, w[1], o);
            }
            if (lane == 0) acc_add_words(L, acc_slot(L, m < 3 ? ACC_FS : ACC_TS, p0, m % 3), w);
        }
    }
}

template <int PREC>
size_t virtual_smem() {
    typedef typename Prec<PREC>::C C;
    return (size_t)(VZC + 2) * (VTY + 2) * (VTX + 2) * (sizeof(int) + 2 * sizeof(C));
}

// -------------------------------------------------------- pair forces
// Eq. 26 (Hertz, repulsive, r floored at r_cap) and Eq. 27 (lubrication) on
// particle i due to j, in FP64.
__device__ void pair_force(const Lattice& L, int i, int j, const double (&ri)[3], double Ri,
                           const double (&vi)[3], double nu, double (&fo)[3]) {
    double rij[3];
    for (int d = 0; d < 3; d++) {
        double dd = L.pos[3 * j + d] - ri[d];
        if (L.per[d]) {
            double Ld = (d == 0 ? L.nx : (d == 1 ? L.ny : L.nz));
            dd -= Ld * floor(dd / Ld + 0.5);
        }
        rij[d] = dd;
    }
    fo[0] = fo[1] = fo[2] = 0.0;
    double r = sqrt(rij[0] * rij[0] + rij[1] * rij[1] + rij[2] * rij[2]);
    if (!(r > 0.0)) return;
    if (L.P.hertz_K != 0.0 && r < L.P.hertz_sigma) {
        double rr = r < L.P.hertz_rcap ? L.P.hertz_rcap : r;
        double mag = 2.5 * L.P.hertz_K * pow(L.P.hertz_sigma - rr, 1.5);
        for (int d = 0; d < 3; d++) fo[d] += -mag * rij[d] / r;
    }
    if (L.P.lub_on) {
        double Rj = L.rad[j];
        double h = r - (Ri + Rj);
        if (h < L.P.lub_hn) {
            double red = Ri * Rj / (Ri + Rj), vr = 0.0;
            if (h < L.P.lub_hmin) h = L.P.lub_hmin;
            for (int d = 0; d < 3; d++) vr += (vi[d] - L.vel[3 * j + d]) * rij[d] / r;
            double mag = -6.0 * 3.14159265358979323846 * nu * L.P.lub_scale * red * red *
                         (1.0 / h - 1.0 / L.P.lub_hn) * vr;
            for (int d = 0; d < 3; d++) fo[d] += mag * rij[d] / r;
        }
    }
}

struct CellGrid {
    int n[3];         // cells per axis (>= 3 each when used)
    float inv[3];     // cells per lattice unit
    int* count;       // [ncell] counts, reused as fill cursors
    int* start;       // [ncell + 1]
    int* items;       // [nc]
};

__device__ __forceinline__ int cell_coord(float x, float inv, int n) {
    int c = (int)(x * inv);
    return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

// The cell list serves the pair-list build: the cell kernels do nothing in a
// step that keeps the list (flag clear).
__global__ void k_cells_count(Lattice L, CellGrid cg) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L.nc || !*L.vl_flag) return;
    int c0 = cell_coord(float(L.pos[3 * p]), cg.inv[0], cg.n[0]);
    int c1 = cell_coord(float(L.pos[3 * p + 1]), cg.inv[1], cg.n[1]);
    int c2 = cell_coord(float(L.pos[3 * p + 2]), cg.inv[2], cg.n[2]);
    atomicAdd(cg.count + (c0 + cg.n[0] * (c1 + cg.n[1] * c2)), 1);
}

// exclusive scan of the counts (one block); counts are reset to serve as cursors
__global__ void __launch_bounds__(1024) k_cells_scan(CellGrid cg, const int* flag) {
    if (!*flag) return;
    __shared__ int part[1024];
    int nc = cg.n[0] * cg.n[1] * cg.n[2];
    int per = (nc + 1023) / 1024;
    int b = threadIdx.x * per, e = min(nc, b + per);
    int sum = 0;
    for (int c = b; c < e; c++) sum += cg.count[c];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - sum;
    for (int c = b; c < e; c++) {
        cg.start[c] = run;
        run += cg.count[c];
        cg.count[c] = 0;
    }
    if (threadIdx.x == 1023) cg.start[nc] = part[1023];
}

__global__ void k_cells_fill(Lattice L, CellGrid cg) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L.nc || !*L.vl_flag) return;
    int c0 = cell_coord(float(L.pos[3 * p]), cg.inv[0], cg.n[0]);
    int c1 = cell_coord(float(L.pos[3 * p + 1]), cg.inv[1], cg.n[1]);
    int c2 = cell_coord(float(L.pos[3 * p + 2]), cg.inv[2], cg.n[2]);
    int c = c0 + cg.n[0] * (c1 + cg.n[1] * c2);
    cg.items[cg.start[c] + atomicAdd(cg.count + c, 1)] = p;
}

// Pair list (App. A rcut / delr): a particle's neighbours within the list
// radius rl = max(rcut, interaction range) + delr, sorted by index, are kept
// until some particle has moved more than delr / 2 since the build; the pair
// forces then reach only listed pairs.  Every pair within the interaction
// range at any step before the next build was within rl at the build.
__global__ void k_pair_check(Lattice L, double half_skin) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L.nc) return;
    double d2 = 0.0;
    for (int d = 0; d < 3; d++) {
        double dd = L.pos[3 * p + d] - L.vl_ref[3 * p + d];
        if (L.per[d]) {
            double Ld = (d == 0 ? L.nx : (d == 1 ? L.ny : L.nz));
            dd -= Ld * floor(dd / Ld + 0.5);
        }
        d2 += dd * dd;
    }
    if (!(d2 <= half_skin * half_skin)) atomicOr(L.vl_flag, 1);
}

// Build the list of particle i (when the flag is set): candidates from the 27
// neighbouring cells, or among all particles when the grid has fewer than 3
// cells along an axis; more than PAIR_LIST_MAX neighbours is reported as an
// overlap.
__global__ void __launch_bounds__(128) k_pair_list(Lattice L, CellGrid cg, int use_cells, float rl) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.nc || !*L.vl_flag) return;
    if (i == 0) atomicAdd(L.vl_builds, 1ull);
    float rif[3];
    for (int d = 0; d < 3; d++) {
        L.vl_ref[3 * i + d] = L.pos[3 * i + d];
        rif[d] = float(L.pos[3 * i + d]);
    }
    float Lf[3] = {float(L.nx), float(L.ny), float(L.nz)};
    float iLf[3] = {1.f / Lf[0], 1.f / Lf[1], 1.f / Lf[2]};
    int* cand = L.vl_nb + (size_t)i * PAIR_LIST_MAX;
    int nc = 0;
    auto test = [&](int j) {
        if (j == i) return;
        float r2 = 0.f;
        for (int d = 0; d < 3; d++) {
            float df = float(L.pos[3 * j + d]) - rif[d];
            if (L.per[d]) df -= Lf[d] * rintf(df * iLf[d]);
            r2 += df * df;
        }
        if (r2 >= rl * rl) return;
        if (nc < PAIR_LIST_MAX) {
            // insertion keeps the list sorted by j
            int q = nc++;
            while (q > 0 && cand[q - 1] > j) {
                cand[q] = cand[q - 1];
                q--;
            }
            cand[q] = j;
        } else {
            atomicOr(L.flags, FLAG_OVERLAP);
        }
    };
    if (rl > 0.f) {
        if (use_cells) {
            int c0 = cell_coord(rif[0], cg.inv[0], cg.n[0]);
            int c1 = cell_coord(rif[1], cg.inv[1], cg.n[1]);
            int c2 = cell_coord(rif[2], cg.inv[2], cg.n[2]);
            for (int dz = -1; dz <= 1; dz++) {
                int z = c2 + dz;
                if (z < 0 || z >= cg.n[2]) {
                    if (!L.per[2]) continue;
                    z = (z + cg.n[2]) % cg.n[2];
                }
                for (int dy = -1; dy <= 1; dy++) {
                    int y = (c1 + dy + cg.n[1]) % cg.n[1];
                    for (int dx = -1; dx <= 1; dx++) {
                        int x = (c0 + dx + cg.n[0]) % cg.n[0];
                        int c = x + cg.n[0] * (y + cg.n[1] * z);
                        for (int q = cg.start[c]; q < cg.start[c + 1]; q++) test(cg.items[q]);
                    }
                }
            }
        } else {
            for (int j = 0; j < L.nc; j++) test(j);
        }
    }
    L.vl_cnt[i] = nc;
}

// Pair forces on particle i summed over its listed neighbours in index
// order, plus the soft side walls.
__global__ void __launch_bounds__(128) k_pairs(Lattice L) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.nc) return;
    double ri[3], vi[3];
    for (int d = 0; d < 3; d++) {
        ri[d] = L.pos[3 * i + d];
        vi[d] = L.vel[3 * i + d];
    }
    double Ri = L.rad[i];
    double nu = 0.5 * ((L.P.tau[0] - 0.5) / 3.0 + (L.P.tau[1] - 0.5) / 3.0);
    NSum acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    const int n = L.vl_cnt[i];
    const int* nb = L.vl_nb + (size_t)i * PAIR_LIST_MAX;
    for (int q = 0; q < n; q++) {
        double fo[3];
        pair_force(L, i, nb[q], ri, Ri, vi, nu, fo);
        for (int d = 0; d < 3; d++) acc[d].add(fo[d]);
    }
    if (!L.per[2] && L.P.side_wall_k != 0.0) {
        double hlo = ri[2] + 0.5, hhi = (double(L.nz) - 0.5) - ri[2];
        if (hlo < L.P.side_wall_d) acc[2].add(L.P.side_wall_k * (L.P.side_wall_d - hlo));
        if (hhi < L.P.side_wall_d) acc[2].add(-L.P.side_wall_k * (L.P.side_wall_d - hhi));
    }
    for (int d = 0; d < 3; d++) L.Fpair[3 * i + d] = acc[d].value();
}

// --------------------------------------------------------- integrator
// Eq. 33: qdot = 1/2 q (0, w*) written out component-wise
__device__ __forceinline__ void qrate(const double (&q)[4], const double (&w)[3], double (&qd)[4]) {
    qd[0] = 0.5 * (-q[1] * w[0] - q[2] * w[1] - q[3] * w[2]);
    qd[1] = 0.5 * (q[0] * w[0] - q[3] * w[1] + q[2] * w[2]);
    qd[2] = 0.5 * (q[3] * w[0] + q[0] * w[1] - q[1] * w[2]);
    qd[3] = 0.5 * (-q[2] * w[0] + q[1] * w[1] + q[0] * w[2]);
}

// body-frame angular velocity R(q/|q|)^T w, R from Eq. 31
__device__ __forceinline__ void to_body(const double (&q)[4], const double (&w)[3], double (&wb)[3]) {
    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double a = q[0] / nq, b = q[1] / nq, c = q[2] / nq, e = q[3] / nq;
    double R00 = a * a + b * b - c * c - e * e, R01 = 2.0 * (b * c - a * e), R02 = 2.0 * (b * e + a * c);
    double R10 = 2.0 * (b * c + a * e), R11 = a * a - b * b + c * c - e * e, R12 = 2.0 * (c * e - a * b);
    double R20 = 2.0 * (b * e - a * c), R21 = 2.0 * (c * e + a * b), R22 = a * a - b * b - c * c + e * e;
    wb[0] = R00 * w[0] + R10 * w[1] + R20 * w[2];
    wb[1] = R01 * w[0] + R11 * w[1] + R21 * w[2];
    wb[2] = R02 * w[0] + R12 * w[1] + R22 * w[2];
}

// Eq. 35 totals, Eq. 32 leap-frog, Eq. 34 implicit mid-step quaternion
// (iterated until the rate changes by <= 1e-14, at most 20 times); then the
// FP32 snapshot of the new state.  A particle faster than 1/2 lattice unit
// per step is reported (the remap assumes smaller moves).
__global__ void k_integrate(Lattice L) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L.nc) return;
    double F[3], T[3];
    bool first = !L.prev_valid[p];
    // the step's fixed-point sums as FP64 terms
    double* terms[ACC_TERMS] = {L.Fliq, L.Tliq, L.Fd, L.Td, L.Fc, L.Tc, L.Fs, L.Ts};
    for (int t = 0; t < ACC_TERMS; t++)
        for (int d = 0; d < 3; d++) terms[t][3 * p + d] = acc_value(L, acc_slot(L, t, p, d));
    for (int d = 0; d < 3; d++) {
        double fp = first ? L.Fliq[3 * p + d] : L.Fliq_prev[3 * p + d];
        double tp = first ? L.Tliq[3 * p + d] : L.Tliq_prev[3 * p + d];
        F[d] = 0.5 * (fp + L.Fliq[3 * p + d]) + L.Fd[3 * p + d] + L.Fc[3 * p + d] + L.Fs[3 * p + d] +
               L.Fpair[3 * p + d];
        T[d] = 0.5 * (tp + L.Tliq[3 * p + d]) + L.Td[3 * p + d] + L.Tc[3 * p + d] + L.Ts[3 * p + d];
        L.Ftot[3 * p + d] = F[d];
        L.Ttot[3 * p + d] = T[d];
        L.Fliq_prev[3 * p + d] = L.Fliq[3 * p + d];
        L.Tliq_prev[3 * p + d] = L.Tliq[3 * p + d];
    }
    L.prev_valid[p] = 1;
    double m = L.mass[p];
    int Ls[3] = {L.nx, L.ny, L.nz};
    for (int d = 0; d < 3; d++) {
        double v = L.vel[3 * p + d] + F[d] / m;
        double r = L.pos[3 * p + d] + v;
        if (L.per[d]) r = r - double(Ls[d]) * floor(r / double(Ls[d]));
        L.vel[3 * p + d] = v;
        L.pos[3 * p + d] = r;
        if (!(fabs(v) < 0.5)) atomicOr(L.flags, FLAG_NONFINITE);
    }
    if (L.P.rotate) {
        double R = L.rad[p];
        double I = 0.4 * m * R * R;
        double w[3], q[4], wb[3], qd[4], qh[4];
        for (int d = 0; d < 3; d++) w[d] = L.omg[3 * p + d] + T[d] / I;
        for (int d = 0; d < 4; d++) q[d] = L.quat[4 * p + d];
        to_body(q, w, wb);
        qrate(q, wb, qd);
        for (int d = 0; d < 4; d++) qh[d] = q[d] + 0.5 * qd[d];
        for (int it = 0; it < 20; it++) {
            double nd[4], delta = 0.0;
            to_body(qh, w, wb);
            qrate(qh, wb, nd);
            for (int d = 0; d < 4; d++) {
                delta = fmax(delta, fabs(nd[d] - qd[d]));
                qh[d] = q[d] + 0.5 * nd[d];
                qd[d] = nd[d];
            }
            if (delta <= 1e-14) break;
        }
        double nq = 0.0;
        for (int d = 0; d < 4; d++) {
            q[d] = q[d] + qd[d];
            nq += q[d] * q[d];
        }
        nq = sqrt(nq);
        for (int d = 0; d < 3; d++) L.omg[3 * p + d] = w[d];
        for (int d = 0; d < 4; d++) L.quat[4 * p + d] = q[d] / nq;
    }
    for (int d = 0; d < 3; d++) {
        double r = L.pos[3 * p + d];
        int ip = (int)floor(r);
        L.ipos[3 * p + d] = ip;
        L.fsnap[9 * p + d] = float(r - (double)ip);
        L.fsnap[9 * p + 3 + d] = float(L.vel[3 * p + d]);
        L.fsnap[9 * p + 6 + d] = float(L.omg[3 * p + d]);
    }
}

// ---------------------------------------------------------- launchers
#define DISPATCHC(prec, call)                                 \
    switch (prec) {                                           \
        case LB_FP64: { const int P = LB_FP64; call; break; } \
        case LB_FP32: { const int P = LB_FP32; call; break; } \
        default:      { const int P = LB_FP16; call; break; } \
    }

static const dim3 PBLK(BXP, BYP);

int launch_snapshot(const Lattice& L, cudaStream_t st) {
    if (L.nc <= 0) return 0;
    k_snapshot<<<(L.nc + 127) / 128, 128, 0, st>>>(L);
    return 1;
}

int launch_map_initial(const Lattice& L, int prec, int first, int count, cudaStream_t st) {
    if (count <= 0) return 0;
    DISPATCHC(prec, (k_map_initial<P><<<count, PBLK, 0, st>>>(L, first)));
    return 1;
}

int launch_remap(const Lattice& L, int prec, int maxc, cudaStream_t st) {
    if (L.nc <= 0) return 0;
    // the per-particle terms of the step are fixed-point sums of block
    // partials and per-site contributions (acc_add), from zero; the
    // integrator turns them into F_liq, T_liq, F_d, T_d, F_c, T_c, F_s, T_s
    (void)maxc;
    cudaMemsetAsync(L.acc, 0, (size_t)ACC_TERMS * L.maxc * 6 * sizeof(unsigned long long), st);
    cudaMemsetAsync(L.nb_chg, 0, sizeof(int), st);
    const dim3 grid((unsigned)L.nc, REMAP_GROUPS);
    DISPATCHC(prec, (k_remap_classify<P><<<grid, PBLK, 0, st>>>(L)));
    // the refill and the commit of the listed nodes; the per-particle shell
    // scans return at once unless the list overflowed
    const unsigned lg = (unsigned)(2 * device_sms());
    DISPATCHC(prec, (k_remap_create_list<P><<<lg, 128, 0, st>>>(L)));
    DISPATCHC(prec, (k_remap_create<P><<<grid, PBLK, 0, st>>>(L)));
    k_remap_commit_list<<<lg, 128, 0, st>>>(L);
    DISPATCHC(prec, (k_remap_commit<P><<<grid, PBLK, 0, st>>>(L)));
    return 5;
}

int launch_link_classes(const Lattice& L, bool full, cudaStream_t st) {
    if (full) {
        const int bx = L.nx >= 128 ? 128 : ((L.nx + 31) / 32) * 32;
        k_link_classes_all<<<dim3((unsigned)((L.nx + bx - 1) / bx), (unsigned)L.ny, (unsigned)L.nz), bx, 0, st>>>(L);
    } else {
        k_link_classes_changed<<<(unsigned)(4 * device_sms()), 256, 0, st>>>(L);
    }
    return 1;
}

int launch_virtual(const Lattice& L, int prec, int store_terms, cudaStream_t st) {
    if (L.nc <= 0) return 0;
    const int zc = L.nz < VZC ? L.nz : VZC;
    dim3 grid((L.nx + VTX - 1) / VTX, (L.ny + VTY - 1) / VTY, (L.nz + zc - 1) / zc);
    DISPATCHC(prec, (kernel_setup<k_virtual<P>>(VTX * VTY, virtual_smem<P>())));
    DISPATCHC(prec, (k_virtual<P><<<grid, dim3(VTX, VTY), virtual_smem<P>(), st>>>(L, store_terms, zc)));
    return 1;
}

int launch_pairs(const Lattice& L, void* cells, size_t cell_cap, bool force_build, cudaStream_t st) {
    if (L.nc <= 0) return 0;
    // interaction range: Hertz contact, and lubrication up to 2 R_max + h_n
    double rc = L.P.hertz_K != 0.0 ? L.P.hertz_sigma : 0.0;
    if (L.P.lub_on) rc = fmax(rc, 2.0 * L.rmax + L.P.lub_hn);
    if (rc > 0.0) rc = fmax(rc, L.P.rcut);
    float rl = rc > 0.0 ? float(rc + L.P.delr) + 0.05f : 0.f;
    CellGrid cg;
    int Ls[3] = {L.nx, L.ny, L.nz};
    long long ncell = 1;
    int use_cells = rl > 0.f && L.nc > 64;
    for (int d = 0; d < 3; d++) {
        int n = rl > 0.f ? (int)(Ls[d] / rl) : 1;
        if (n > 64) n = 64;
        if (n < 3) use_cells = 0;
        cg.n[d] = n < 1 ? 1 : n;
        cg.inv[d] = float(cg.n[d]) / float(Ls[d]);
        ncell *= cg.n[d];
    }
    if ((size_t)(2 * ncell + 1 + L.nc) * sizeof(int) > cell_cap) use_cells = 0;
    int n = 0;
    cg.count = (int*)cells;
    cg.start = cg.count + ncell;
    cg.items = cg.start + ncell + 1;
    // rebuild flag: forced (new particles or parameters, or no skin), else
    // set by the particles that moved more than delr / 2
    const bool every_step = force_build || !(L.P.delr > 0.0);
    cudaMemsetAsync(L.vl_flag, every_step ? 0xff : 0, sizeof(int), st);
    if (!every_step) {
        k_pair_check<<<(L.nc + 127) / 128, 128, 0, st>>>(L, 0.5 * L.P.delr);
        n++;
    }
    if (use_cells) {
        cudaMemsetAsync(cg.count, 0, ncell * sizeof(int), st);
        k_cells_count<<<(L.nc + 127) / 128, 128, 0, st>>>(L, cg);
        k_cells_scan<<<1, 1024, 0, st>>>(cg, L.vl_flag);
        k_cells_fill<<<(L.nc + 127) / 128, 128, 0, st>>>(L, cg);
        n += 3;
    }
    k_pair_list<<<(L.nc + 127) / 128, 128, 0, st>>>(L, cg, use_cells, rl);
    k_pairs<<<(L.nc + 127) / 128, 128, 0, st>>>(L);
    return n + 2;
}

int launch_integrate(const Lattice& L, cudaStream_t st) {
    if (L.nc <= 0) return 0;
    k_integrate<<<(L.nc + 127) / 128, 128, 0, st>>>(L);
    return 1;
}

}  // namespace lbgb
