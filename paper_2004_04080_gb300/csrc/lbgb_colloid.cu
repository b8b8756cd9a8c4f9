// lbgb_colloid.cu -- particle kernels: node map and remap (destroy / create),
// wetting virtual densities with the solid-node Shan-Chen force, Ladd link
// forces, pair forces and the rotational leap-frog integrator.
//
// Per-particle work runs one thread block per particle over a box around the
// sphere; every per-particle sum is a Neumaier-compensated FP64 sum, reduced
// in a fixed order (each thread's fixed share of the box, then warp shuffles,
// then warps in order), so the result does not depend on scheduling.
#include "lbgb_internal.cuh"

namespace lbgb {

constexpr int PB = 128;  // threads per particle block

// box of lattice points around particle p, padded by `pad`
struct PBox {
    int lo[3], ext[3], total;
    double r[3], R;
};

__device__ __forceinline__ PBox make_box(const Lattice& L, int p, double pad) {
    PBox b;
    b.R = L.rad[p];
    b.total = 1;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        b.r[d] = L.pos[3 * p + d];
        int lo = (int)floor(b.r[d] - b.R - pad);
        int hi = (int)ceil(b.r[d] + b.R + pad);
        b.lo[d] = lo;
        b.ext[d] = hi - lo + 1;
        b.total *= b.ext[d];
    }
    return b;
}

// t-th point of the box: wrapped site (X,Y,Z), offset d = point - r_p (no
// wrap needed: the box is smaller than half of every periodic side).
// Returns false for points beyond a wall.
__device__ __forceinline__ bool box_point(const Lattice& L, const PBox& b, int t, int& X, int& Y,
                                          int& Z, double (&d)[3]) {
    int a = b.lo[0] + t % b.ext[0];
    int c = b.lo[1] + (t / b.ext[0]) % b.ext[1];
    int e = b.lo[2] + t / (b.ext[0] * b.ext[1]);
    d[0] = (double)a - b.r[0];
    d[1] = (double)c - b.r[1];
    d[2] = (double)e - b.r[2];
    if (!L.per[2] && (e < 0 || e >= L.nz)) return false;
    X = ((a % L.nx) + L.nx) % L.nx;
    Y = ((c % L.ny) + L.ny) % L.ny;
    Z = ((e % L.nz) + L.nz) % L.nz;
    return true;
}

// |d|^2 without fused multiply-add, so that node membership (|d|^2 < R^2) is
// decided with the same rounding as a plain double evaluation
__device__ __forceinline__ double dist2(const double (&d)[3]) {
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

__device__ __forceinline__ void crossd(const double (&a)[3], const double (&b)[3], double (&o)[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ long long sidx(const Lattice& L, int X, int Y, int Z) {
    return (long long)X + (long long)L.nx * ((long long)Y + (long long)L.ny * Z);
}

// Block-wide deterministic reduction of M compensated sums; thread 0 gets
// the results in out[0..M-1].
template <int M>
__device__ void block_reduce(NSum (&acc)[M], double* out) {
    __shared__ double sh_s[PB / 32][M], sh_c[PB / 32][M];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int m = 0; m < M; m++) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            NSum o;
            o.s = __shfl_down_sync(0xffffffffu, acc[m].s, off);
            o.c = __shfl_down_sync(0xffffffffu, acc[m].c, off);
            if (lane < off) acc[m].merge(o);
        }
        if (lane == 0) {
            sh_s[warp][m] = acc[m].s;
            sh_c[warp][m] = acc[m].c;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int m = 0; m < M; m++) {
            NSum t = {sh_s[0][m], sh_c[0][m]};
            for (int w = 1; w < PB / 32; w++) {
                NSum o = {sh_s[w][m], sh_c[w][m]};
                t.merge(o);
            }
            out[m] = t.value();
        }
    }
}

// density of component k at a site from its populations (same order as the
// lattice kernels)
template <int PREC>
__device__ __forceinline__ typename Prec<PREC>::C site_rho(const Lattice& L, long long s, int k) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    const S* f = (const S*)L.f_cur;
    C r = 0;
#pragma unroll
    for (int i = 0; i < Q; i++)
        r += ld_pop(f + ((long long)(k * Q + i)) * L.pstride + s, pop_shift<S, C>(L, k, i));
    return r;
}

// ------------------------------------------------------ initial node map
// First map after particles are added: solid nodes are claimed without
// momentum bookkeeping (Sec. 2.4).
__global__ void __launch_bounds__(PB) k_map_initial(Lattice L, int first) {
    int p = first + blockIdx.x;
    PBox b = make_box(L, p, 0.0);
    for (int t = threadIdx.x; t < b.total; t += PB) {
        int X, Y, Z;
        double d[3];
        if (!box_point(L, b, t, X, Y, Z, d)) continue;
        if (!(dist2(d) < b.R * b.R)) continue;
        long long s = sidx(L, X, Y, Z);
        int old = atomicCAS(L.owner + s, -1, p);
        if (old != -1 && old != p) atomicOr(L.flags, FLAG_OVERLAP);
        L.mask[s] = 1;
    }
}

// ------------------------------------------------------------- remap
// Classify the nodes around particle p at its new position r_p(t):
//   fluid node now inside  -> destroy (Eq. 24): its momentum rho u goes to p
//   node of p now outside  -> create (handled by k_remap_create)
template <int PREC>
__global__ void __launch_bounds__(PB) k_remap_classify(Lattice L) {
    typedef typename Prec<PREC>::C C;
    int p = blockIdx.x;
    PBox b = make_box(L, p, 2.0);
    NSum acc[6];
#pragma unroll
    for (int m = 0; m < 6; m++) acc[m].s = acc[m].c = 0.0;
    for (int t = threadIdx.x; t < b.total; t += PB) {
        int X, Y, Z;
        double d[3];
        if (!box_point(L, b, t, X, Y, Z, d)) continue;
        long long s = sidx(L, X, Y, Z);
        bool inside = dist2(d) < b.R * b.R;
        int o = L.owner[s];
        if (inside) {
            if (o == -1) {
                int prev = atomicCAS(L.evt + s, 0, 4 * (p + 1) + 1);
                if (prev != 0) {
                    atomicOr(L.flags, FLAG_OVERLAP);
                    continue;
                }
                C fv[2][Q], rho[2], j[2][3], u[3], om;
                load_site<PREC>(L, (const typename Prec<PREC>::S*)L.f_cur, s, fv, rho, j);
                mixture<C>(L, rho, j, u, om);
                double rt = double(rho[0] + rho[1]);
                double mom[3] = {rt * double(u[0]), rt * double(u[1]), rt * double(u[2])}, tq[3];
                crossd(d, mom, tq);
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
        }
    }
    double out[6];
    block_reduce<6>(acc, out);
    if (threadIdx.x == 0)
        for (int m = 0; m < 3; m++) {
            L.Fd[3 * p + m] = out[m];
            L.Td[3 * p + m] = out[3 + m];
        }
}

// Refill the nodes released by p (Eq. 25): f = f^eq(rhobar^k, u_w) with
// rhobar^k the w_i-weighted mean over neighbours that are fluid before and
// after the remap, u_w = v_p + omega_p x (r - r_p); p loses (rhobar) u_w.
template <int PREC>
__global__ void __launch_bounds__(PB) k_remap_create(Lattice L) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    int p = blockIdx.x;
    PBox b = make_box(L, p, 2.0);
    NSum acc[6];
#pragma unroll
    for (int m = 0; m < 6; m++) acc[m].s = acc[m].c = 0.0;
    const int code = 4 * (p + 1) + 2;
    for (int t = threadIdx.x; t < b.total; t += PB) {
        int X, Y, Z;
        double d[3];
        if (!box_point(L, b, t, X, Y, Z, d)) continue;
        long long s = sidx(L, X, Y, Z);
        if (L.evt[s] != code) continue;
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
        const double* v = L.vel + 3 * p;
        const double* w = L.omg + 3 * p;
        double uw[3] = {v[0] + (w[1] * d[2] - w[2] * d[1]), v[1] + (w[2] * d[0] - w[0] * d[2]),
                        v[2] + (w[0] * d[1] - w[1] * d[0])};
        C ux = C(uw[0]), uy = C(uw[1]), uz = C(uw[2]);
        C uu = ux * ux + uy * uy + uz * uz;
        S* f = (S*)L.f_cur;
        for (int k = 0; k < 2; k++)
            for (int i = 0; i < Q; i++)
                st_pop(f + ((long long)(k * Q + i)) * L.pstride + s, feq<C>(i, rb[k], ux, uy, uz, uu),
                       pop_shift<S, C>(L, k, i));
        double rt = double(rb[0] + rb[1]);
        double mom[3] = {-rt * uw[0], -rt * uw[1], -rt * uw[2]}, tq[3];
        crossd(d, mom, tq);
#pragma unroll
        for (int m = 0; m < 3; m++) {
            acc[m].add(mom[m]);
            acc[3 + m].add(tq[m]);
        }
    }
    double out[6];
    block_reduce<6>(acc, out);
    if (threadIdx.x == 0)
        for (int m = 0; m < 3; m++) {
            L.Fc[3 * p + m] = out[m];
            L.Tc[3 * p + m] = out[3 + m];
        }
}

// Commit the new node map of particle p.
__global__ void __launch_bounds__(PB) k_remap_commit(Lattice L) {
    int p = blockIdx.x;
    PBox b = make_box(L, p, 2.0);
    for (int t = threadIdx.x; t < b.total; t += PB) {
        int X, Y, Z;
        double d[3];
        if (!box_point(L, b, t, X, Y, Z, d)) continue;
        long long s = sidx(L, X, Y, Z);
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
    }
}

// ------------------------------------------------------------ wetting
// Eq. 20 on each frontier node s of particle p (a node of p with at least one
// fluid neighbour): psi^k(s) = (1 + zeta^k) sum w_i rho^k / sum w_i over fluid
// neighbours; and Eq. 21 (repulsive sign): F_s = -G sum_k psi^k(s) sum w_i
// rho^kbar(s + c_i) c_i over fluid neighbours, summed with its torque.
template <int PREC>
__global__ void __launch_bounds__(PB) k_virtual(Lattice L, int store_terms) {
    typedef typename Prec<PREC>::C C;
    int p = blockIdx.x;
    PBox b = make_box(L, p, 0.0);
    C* psi = (C*)L.psi;
    NSum acc[6];
#pragma unroll
    for (int m = 0; m < 6; m++) acc[m].s = acc[m].c = 0.0;
    for (int t = threadIdx.x; t < b.total; t += PB) {
        int X, Y, Z;
        double d[3];
        if (!box_point(L, b, t, X, Y, Z, d)) continue;
        long long s = sidx(L, X, Y, Z);
        if (L.owner[s] != p) continue;
        SiteNbr n = site_nbr(L, X, Y, Z);
        C num[2] = {0, 0}, den = 0;
        C sA[3] = {0, 0, 0}, sB[3] = {0, 0, 0};
        for (int i = 1; i < Q; i++) {
            if (nbr_is_wall(n, i)) continue;
            long long m = nbr_index(L, n, i);
            if (L.mask[m]) continue;
            C w = wgt<C>(i);
            C ra = psi[m], rb = psi[L.N + m];
            num[0] += w * ra;
            num[1] += w * rb;
            den += w;
            sA[0] += w * ra * C(cx(i)); sA[1] += w * ra * C(cy(i)); sA[2] += w * ra * C(cz(i));
            sB[0] += w * rb * C(cx(i)); sB[1] += w * rb * C(cy(i)); sB[2] += w * rb * C(cz(i));
        }
        if (!(den > C(0))) continue;
        C pa = (C(1) + C(L.P.zeta[0])) * num[0] / den;
        C pb = (C(1) + C(L.P.zeta[1])) * num[1] / den;
        psi[s] = pa;
        psi[L.N + s] = pb;
        if (store_terms) {
            C G = C(L.P.G);
            double fs[3], tq[3];
            for (int m = 0; m < 3; m++) fs[m] = double(-G * pa * sB[m]) + double(-G * pb * sA[m]);
            crossd(d, fs, tq);
#pragma unroll
            for (int m = 0; m < 3; m++) {
                acc[m].add(fs[m]);
                acc[3 + m].add(tq[m]);
            }
        }
    }
    if (!store_terms) return;
    double out[6];
    block_reduce<6>(acc, out);
    if (threadIdx.x == 0)
        for (int m = 0; m < 3; m++) {
            L.Fs[3 * p + m] = out[m];
            L.Ts[3 * p + m] = out[3 + m];
        }
}

// ------------------------------------------------------------- links
// Eq. 19 on every link (x, i) from a fluid node x to a node of p:
// F_i = [2 f*_i(x) - 2 w_i rho^k (u_w.c_i)/cs^2] c_i summed over k, with
// f*_i(x) recovered from the bounced population f_ibar(x, t+1) written by the
// lattice step; Eqs. 22-23 sum the forces and torques (r_w - r_p) x F_i.
template <int PREC>
__global__ void __launch_bounds__(PB) k_links(Lattice L) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    int p = blockIdx.x;
    PBox b = make_box(L, p, 2.0);
    const C* psi = (const C*)L.psi;
    const S* fn = (const S*)L.f_nxt;
    const double* v = L.vel + 3 * p;
    const double* w = L.omg + 3 * p;
    NSum acc[6];
#pragma unroll
    for (int m = 0; m < 6; m++) acc[m].s = acc[m].c = 0.0;
    for (int t = threadIdx.x; t < b.total; t += PB) {
        int X, Y, Z;
        double d[3];
        if (!box_point(L, b, t, X, Y, Z, d)) continue;
        long long s = sidx(L, X, Y, Z);
        if (L.mask[s]) continue;
        SiteNbr n = site_nbr(L, X, Y, Z);
        C rho0 = psi[s], rho1 = psi[L.N + s];
        for (int i = 1; i < Q; i++) {
            if (nbr_is_wall(n, i)) continue;
            long long m = nbr_index(L, n, i);
            if (L.owner[m] != p) continue;
            double rel[3] = {d[0] + 0.5 * cx(i), d[1] + 0.5 * cy(i), d[2] + 0.5 * cz(i)};
            double uw[3] = {v[0] + (w[1] * rel[2] - w[2] * rel[1]),
                            v[1] + (w[2] * rel[0] - w[0] * rel[2]),
                            v[2] + (w[0] * rel[1] - w[1] * rel[0])};
            C cu = C(cx(i) * uw[0] + cy(i) * uw[1] + cz(i) * uw[2]);
            int ib = opp(i);
            double fl = 0.0;
            for (int k = 0; k < 2; k++) {
                C corr = C(6) * wgt<C>(i) * (k == 0 ? rho0 : rho1) * cu;
                C fstar = ld_pop(fn + ((long long)(k * Q + ib)) * L.pstride + s, pop_shift<S, C>(L, k, ib)) + corr;
                fl += double(C(2) * fstar - corr);
            }
            double F[3] = {fl * cx(i), fl * cy(i), fl * cz(i)}, tq[3];
            crossd(rel, F, tq);
#pragma unroll
            for (int q = 0; q < 3; q++) {
                acc[q].add(F[q]);
                acc[3 + q].add(tq[q]);
            }
        }
    }
    double out[6];
    block_reduce<6>(acc, out);
    if (threadIdx.x == 0)
        for (int m = 0; m < 3; m++) {
            L.Fliq[3 * p + m] = out[m];
            L.Tliq[3 * p + m] = out[3 + m];
        }
}

// -------------------------------------------------------- pair forces
// Eq. 26 (Hertz, repulsive, r floored at r_cap) and Eq. 27 (lubrication) on
// particle i, summed over j in index order, plus the soft side walls.
// Candidates are found with an FP32 distance test on positions staged in
// shared memory; each candidate force is then evaluated in FP64.
constexpr int PT = 128;
__global__ void __launch_bounds__(PT) k_pairs(Lattice L) {
    __shared__ float sp[PT][3];
    int i = blockIdx.x * PT + threadIdx.x;
    bool act = i < L.nc;
    double ri[3] = {0, 0, 0}, vi[3] = {0, 0, 0}, Ri = 0;
    if (act)
        for (int d = 0; d < 3; d++) {
            ri[d] = L.pos[3 * i + d];
            vi[d] = L.vel[3 * i + d];
        }
    if (act) Ri = L.rad[i];
    float rif[3] = {float(ri[0]), float(ri[1]), float(ri[2])};
    float Ls[3] = {float(L.nx), float(L.ny), float(L.nz)};
    double rc = L.P.hertz_K != 0.0 ? L.P.hertz_sigma : 0.0;
    if (L.P.lub_on) rc = fmax(rc, 2.0 * L.rmax + L.P.lub_hn);
    float rcf = float(rc) + 0.05f;
    NSum acc[3];
    for (int m = 0; m < 3; m++) acc[m].s = acc[m].c = 0.0;
    double nu = 0.5 * ((L.P.tau[0] - 0.5) / 3.0 + (L.P.tau[1] - 0.5) / 3.0);
    for (int base = 0; base < L.nc; base += PT) {
        int jj = base + threadIdx.x;
        if (jj < L.nc)
            for (int d = 0; d < 3; d++) sp[threadIdx.x][d] = float(L.pos[3 * jj + d]);
        __syncthreads();
        int cnt = min(PT, L.nc - base);
        if (act && rc > 0.0) {
            for (int q = 0; q < cnt; q++) {
                int j = base + q;
                if (j == i) continue;
                float df[3], r2f = 0.f;
                for (int d = 0; d < 3; d++) {
                    df[d] = sp[q][d] - rif[d];
                    if (L.per[d]) df[d] -= Ls[d] * rintf(df[d] / Ls[d]);
                    r2f += df[d] * df[d];
                }
                if (r2f >= rcf * rcf) continue;
                double rij[3];
                for (int d = 0; d < 3; d++) {
                    double dd = L.pos[3 * j + d] - ri[d];
                    if (L.per[d]) {
                        double Ld = (d == 0 ? L.nx : (d == 1 ? L.ny : L.nz));
                        dd -= Ld * floor(dd / Ld + 0.5);
                    }
                    rij[d] = dd;
                }
                double r = sqrt(rij[0] * rij[0] + rij[1] * rij[1] + rij[2] * rij[2]);
                if (!(r > 0.0)) continue;
                double fo[3] = {0, 0, 0};
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
                for (int d = 0; d < 3; d++) acc[d].add(fo[d]);
            }
        }
        __syncthreads();
    }
    if (!act) return;
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
// (iterated until the rate changes by <= 1e-14, at most 20 times).
__global__ void k_integrate(Lattice L) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L.nc) return;
    double F[3], T[3];
    bool first = !L.prev_valid[p];
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
    }
    if (!L.P.rotate) return;
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

// ---------------------------------------------------------- launchers
#define DISPATCHC(prec, call)                                 \
    switch (prec) {                                           \
        case LB_FP64: { const int P = LB_FP64; call; break; } \
        case LB_FP32: { const int P = LB_FP32; call; break; } \
        default:      { const int P = LB_FP16; call; break; } \
    }

int launch_map_initial(const Lattice& L, int first, int count, cudaStream_t st) {
    if (count <= 0) return 0;
    k_map_initial<<<count, PB, 0, st>>>(L, first);
    return 1;
}

int launch_remap(const Lattice& L, int prec, cudaStream_t st) {
    if (L.nc <= 0) return 0;
    DISPATCHC(prec, (k_remap_classify<P><<<L.nc, PB, 0, st>>>(L)));
    DISPATCHC(prec, (k_remap_create<P><<<L.nc, PB, 0, st>>>(L)));
    k_remap_commit<<<L.nc, PB, 0, st>>>(L);
    return 3;
}

int launch_virtual(const Lattice& L, int prec, int store_terms, cudaStream_t st) {
    if (L.nc <= 0) return 0;
    DISPATCHC(prec, (k_virtual<P><<<L.nc, PB, 0, st>>>(L, store_terms)));
    return 1;
}

int launch_links(const Lattice& L, int prec, cudaStream_t st) {
    if (L.nc <= 0) return 0;
    DISPATCHC(prec, (k_links<P><<<L.nc, PB, 0, st>>>(L)));
    return 1;
}

int launch_pairs_integrate(const Lattice& L, cudaStream_t st) {
    if (L.nc <= 0) return 0;
    k_pairs<<<(L.nc + PT - 1) / PT, PT, 0, st>>>(L);
    k_integrate<<<(L.nc + 127) / 128, 128, 0, st>>>(L);
    return 2;
}

}  // namespace lbgb
