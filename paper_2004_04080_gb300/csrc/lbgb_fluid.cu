// lbgb_fluid.cu -- lattice kernels: initialisation, densities, the fused
// collide + Shan-Chen + bounce-back + push-stream step, and read-outs.
//
// Populations are stored per link plane as component pairs: link i of site
// s = x + nx (y + ny z) is the pair SKEW + s - c_ix of plane i (pair_index),
// both components side by side.  The state between time steps is the post-streaming
// population f(t) (the paper's step starts from it, Sec. 3.1); one step
// reads f(t) at each site, collides locally and pushes f*(t) to the
// neighbours, writing f(t+1) into the second buffer.
#include <cuda.h>
#include <stddef.h>

#include <type_traits>

#include "lbgb_internal.cuh"

namespace lbgb {

// -------------------------------------------------------------- kernels
template <int PREC>
__global__ void k_init(Lattice L, const double* __restrict__ stage) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= L.N) return;
    C ux = C(stage[2 * L.N + s]), uy = C(stage[3 * L.N + s]), uz = C(stage[4 * L.N + s]);
    C uu = ux * ux + uy * uy + uz * uz;
    S* f = (S*)L.f_cur;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        C r = C(stage[k * L.N + s]);
#pragma unroll
        for (int i = 0; i < Q; i++)
            st_pop(f + pop_index(k * Q + i, s, L.pstride), feq<C>(i, r, ux, uy, uz, uu), pop_shift<S, C>(L, k, i));
    }
}

// rho^k on fluid nodes (0 on particle nodes) into psi; flags non-finite or
// negative densities.  MOM: also the total momentum j^A + j^B (Eq. 7) into
// the rows mom[d][s] (0 on particle nodes), for the omega = 1 collision: with
// tau_A = tau_B the mixture velocity (Eq. 14) needs only the sum.
template <int PREC, bool MOM>
__global__ void k_density(Lattice L) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= L.N) return;
    C* psi = (C*)L.psi;
    C* mom = (C*)L.mom;
    if (L.mask[s]) {
        psi[2 * s] = 0;
        psi[2 * s + 1] = 0;
        if (MOM)
#pragma unroll
            for (int a = 0; a < 3; a++) mom[a * L.pstride + s] = 0;
        return;
    }
    const S* f = (const S*)L.f_cur;
    C rho[2] = {0, 0}, jt[2][3] = {{0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int i = 0; i < Q; i++) {
        C v[2];
        ld_pair(f + pair_index(i, s, L.pstride), pop_shift<S, C>(L, 0, i), pop_shift<S, C>(L, 1, i), v[0], v[1]);
#pragma unroll
        for (int k = 0; k < 2; k++) {
            rho[k] += v[k];
            if (MOM) {
                if (cx(i) > 0) jt[k][0] += v[k]; else if (cx(i) < 0) jt[k][0] -= v[k];
                if (cy(i) > 0) jt[k][1] += v[k]; else if (cy(i) < 0) jt[k][1] -= v[k];
                if (cz(i) > 0) jt[k][2] += v[k]; else if (cz(i) < 0) jt[k][2] -= v[k];
            }
        }
    }
    psi[2 * s] = rho[0];
    psi[2 * s + 1] = rho[1];
    if (MOM)
#pragma unroll
        for (int d = 0; d < 3; d++) mom[d * L.pstride + s] = jt[0][d] + jt[1][d];
    if (!(rho[0] >= C(0) && rho[1] >= C(0) && rho[0] < C(1e30) && rho[1] < C(1e30)))
        atomicOr(L.flags, FLAG_NONFINITE);
}

// wall density ("wetting mode 0"): w_i-weighted mean density of the fluid
// neighbours of the wall node below z = 0 (side 0) or above z = nz-1 (side 1)
template <typename C>
__global__ void k_wall_psi(Lattice L) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    int side = blockIdx.z;
    if (x >= L.nx) return;
    const C* psi = (const C*)L.psi;
    C* pw = (C*)L.psi_wall;
    int zf = side == 0 ? 0 : L.nz - 1;
    int dz = side == 0 ? 1 : -1;
    long long nxy = (long long)L.nx * L.ny;
    C num0 = 0, num1 = 0, den = 0;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        if (cz(i) != dz) continue;
        int X = x + cx(i), Y = y + cy(i);
        X = X < 0 ? X + L.nx : (X >= L.nx ? X - L.nx : X);
        Y = Y < 0 ? Y + L.ny : (Y >= L.ny ? Y - L.ny : Y);
        long long m = (long long)X + (long long)L.nx * ((long long)Y + (long long)L.ny * zf);
        if (L.mask[m]) continue;
        C w = wgt<C>(i);
        num0 += w * psi[2 * m];
        num1 += w * psi[2 * m + 1];
        den += w;
    }
    long long w = (long long)x + (long long)L.nx * y;
    const bool face = L.P.open[side] == 1 || L.P.open[side] == 3;  // a pressure or equilibrium face
    pw[2 * (side * nxy + w)] = face ? C(L.P.open_rho[side][0]) : (den > C(0) ? num0 / den : C(0));
    pw[2 * (side * nxy + w) + 1] = face ? C(L.P.open_rho[side][1]) : (den > C(0) ? num1 / den : C(0));
}

// rho^k and the mixture velocity u (Eqs. 6, 7, 14) of fluid node s from f(t)
template <int PREC>
__device__ __forceinline__ void node_values(const Lattice& L, long long s, typename Prec<PREC>::C (&q)[5]) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    const S* f = (const S*)L.f_cur;
    C rho[2] = {0, 0}, j[2][3] = {{0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int i = 0; i < Q; i++) {
        C v[2];
        ld_pair(f + pair_index(i, s, L.pstride), pop_shift<S, C>(L, 0, i), pop_shift<S, C>(L, 1, i), v[0], v[1]);
#pragma unroll
        for (int k = 0; k < 2; k++) {
            rho[k] += v[k];
            j[k][0] += C(cx(i)) * v[k];
            j[k][1] += C(cy(i)) * v[k];
            j[k][2] += C(cz(i)) * v[k];
        }
    }
    C u[3], om;
    mixture<C>(L, rho, j, u, om);
    q[0] = rho[0];
    q[1] = rho[1];
#pragma unroll
    for (int d = 0; d < 3; d++) q[2 + d] = u[d];
}

// The face values of the open z faces with extrapolation (Sec. 2.2), one
// thread per column (x, y) of face blockIdx.z: rho_w^k and u_w at the face
// plane, q_w = q_b + (q_b - q_{b+1}) / 2 from the boundary node b and the
// next interior node b + 1 along z; q_b alone where b + 1 is a particle node
// or nz < 2.  From f(t) after the remap, like every lattice kernel of the
// step.  The face rules read rho_w of velocity faces (Eq. 9) and u_w of
// pressure faces (Eq. 10) from here.
template <int PREC>
__global__ void k_face_values(Lattice L) {
    typedef typename Prec<PREC>::C C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, side = blockIdx.z;
    const int type = L.P.open[side];
    if (x >= L.nx || (type != 1 && type != 2)) return;
    const long long nxy = (long long)L.nx * L.ny, col = (long long)x + (long long)L.nx * y;
    const int zb = side == 0 ? 0 : L.nz - 1, zi = side == 0 ? 1 : L.nz - 2;
    const long long b = col + nxy * zb;
    if (L.mask[b]) return;  // a particle node on the face keeps what it holds
    C q[5];
    node_values<PREC>(L, b, q);
    if (zi >= 0 && zi < L.nz && !L.mask[col + nxy * zi]) {
        C qi[5];
        node_values<PREC>(L, col + nxy * zi, qi);
#pragma unroll
        for (int a = 0; a < 5; a++) q[a] += C(0.5) * (q[a] - qi[a]);
    }
    C* fv = (C*)L.face + 5 * (side * nxy + col);
#pragma unroll
    for (int a = 0; a < 5; a++) fv[a] = q[a];
}

// Add the link force and torque of one site (Eqs. 22, 23) to the fixed-point
// sums of F_liq, T_liq of its particle (p < 0: no link of the site reaches a
// particle).  Integer atomics: the sums do not depend on the order of the
// additions, so they are the same bits on every run.
template <typename C>
__device__ __forceinline__ void commit_link_forces(const Lattice& L, int p, const C (&F)[3], const C (&T)[3]) {
    if (p < 0) return;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        acc_add(L, acc_slot(L, ACC_FLIQ, p, d), F[d]);
        acc_add(L, acc_slot(L, ACC_TLIQ, p, d), T[d]);
    }
}

// ------------------------------------------------------- fused step
// One launch performs the whole lattice update of a time step (Sec. 3.1,
// steps 1, 4-6, 8) for the fluid: each block owns a 32 x 8 column of sites
// and marches along z through a chunk of planes.  Per plane it
//   1. loads the 2 x 19 populations f(t) of its own sites (kept in registers
//      for the next iteration) and forms rho^k (Eq. 6) and j^k (Eq. 7);
//   2. takes rho^k of the one-site ring around the tile: with particles
//      present from the full density pass that precedes the virtual
//      densities (Eq. 20) of the particle nodes; without particles from the
//      ring's populations (these loads mostly hit L2: the neighbouring blocks
//      read the same lines), so that no separate density pass is needed.
//      Particle nodes contribute their virtual density and wall planes the
//      wall density, both precomputed by small kernels;
//   3. keeps psi^k of three consecutive planes (tile + ring) in shared
//      memory, from which the previous plane's Shan-Chen force (Eq. 11) is
//      taken, then collides it (Eqs. 14-16) and pushes f*(t) to the
//      neighbours (Eq. 3), bouncing back on particle and wall links
//      (Eqs. 9, 17, 18).
constexpr int FTX = 32, FTY = 8, FNT = FTX * FTY;
constexpr int RW = FTX + 2, RH = FTY + 2;

// shared state of one block: psi^k and node flags of three planes (tile +
// ring) and the raw populations of the own sites of the plane being collided

template <int PREC>
struct FusedShared {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    C psi[3][2][RH][RW];
    int nd[3][RH][RW];
    S stage[2 * Q][FNT];
};

template <int PREC>
struct OwnSite {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    S raw[2 * Q];  // populations as stored
    C rho[2];
    C j[2][3];
};

template <int PREC>
__device__ __forceinline__ void own_moments(const Lattice& L, OwnSite<PREC>& o) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        C r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            C v = ld_pop(&o.raw[k * Q + i], pop_shift<S, C>(L, k, i));
            r += v;
            if (cx(i) > 0) jx += v; else if (cx(i) < 0) jx -= v;
            if (cy(i) > 0) jy += v; else if (cy(i) < 0) jy -= v;
            if (cz(i) > 0) jz += v; else if (cz(i) < 0) jz -= v;
        }
        o.rho[k] = r;
        o.j[k][0] = jx; o.j[k][1] = jy; o.j[k][2] = jz;
    }
}

// Fill shared slot `slot` with plane zp: psi^k and node flags of the tile and
// its ring.  The calling thread's own site is loaded into `own` (returns
// true if it is a fluid node whose populations were loaded).
template <int PREC>
__device__ __forceinline__ bool fill_plane(const Lattice& L, FusedShared<PREC>& sh, int slot, int zp, int x0,
                                           int y0, int W, int H, bool want_own, OwnSite<PREC>& own) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    const S* f = (const S*)L.f_cur;
    const C* psi = (const C*)L.psi;
    int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FTX + tx;
    bool loaded = false;
    if ((zp < 0 || zp >= L.nz) && !L.per[2]) {
        // a wall plane: the wall density of every tile + ring position
        const C* pw = (const C*)L.psi_wall;
        int side = zp < 0 ? 0 : 1;
        long long nxy = (long long)L.nx * L.ny;
        for (int q = tid; q < (W + 2) * (H + 2); q += FNT) {
            int lx = q % (W + 2) - 1, ly = q / (W + 2) - 1;
            int X = x0 + lx, Y = y0 + ly;
            X = X < 0 ? X + L.nx : (X >= L.nx ? X - L.nx : X);
            Y = Y < 0 ? Y + L.ny : (Y >= L.ny ? Y - L.ny : Y);
            long long w = (long long)X + (long long)L.nx * Y;
            sh.psi[slot][0][ly + 1][lx + 1] = pw[2 * (side * nxy + w)];
            sh.psi[slot][1][ly + 1][lx + 1] = pw[2 * (side * nxy + w) + 1];
            sh.nd[slot][ly + 1][lx + 1] = ND_WALL;
        }
        return false;
    }
    int Z = zp < 0 ? zp + L.nz : (zp >= L.nz ? zp - L.nz : zp);
    long long zoff = (long long)L.nx * L.ny * Z;
    if (tx < W && ty < H) {
        long long s = (long long)(x0 + tx) + (long long)L.nx * (y0 + ty) + zoff;
        if (L.mask[s]) {
            sh.psi[slot][0][ty + 1][tx + 1] = psi[2 * s];
            sh.psi[slot][1][ty + 1][tx + 1] = psi[2 * s + 1];
            sh.nd[slot][ty + 1][tx + 1] = L.owner[s];
            // a particle node collides on finite placeholder moments (its
            // stores write the rest equilibrium)
#pragma unroll
            for (int k = 0; k < 2; k++) {
                own.rho[k] = prm<C>(L.P.rho0[k], L.PF.rho0[k]);
                own.j[k][0] = own.j[k][1] = own.j[k][2] = C(0);
            }
            if (want_own)
#pragma unroll
                for (int q = 0; q < 2 * Q; q++) own.raw[q] = S(0);
            loaded = want_own;
        } else {
            if (want_own) {
#pragma unroll
                for (int q = 0; q < 2 * Q; q++) own.raw[q] = f[pop_index(q, s, L.pstride)];
                own_moments<PREC>(L, own);
                loaded = true;
            } else {
#pragma unroll
                for (int k = 0; k < 2; k++) {
                    C r = 0;
#pragma unroll
                    for (int i = 0; i < Q; i++)
                        r += ld_pop(f + pop_index(k * Q + i, s, L.pstride), pop_shift<S, C>(L, k, i));
                    own.rho[k] = r;
                }
            }
            sh.psi[slot][0][ty + 1][tx + 1] = own.rho[0];
            sh.psi[slot][1][ty + 1][tx + 1] = own.rho[1];
            sh.nd[slot][ty + 1][tx + 1] = ND_FLUID;
        }
    }
    // ring: rows ly = -1 and ly = H (lx = -1..W), columns lx = -1 and lx = W (ly = 0..H-1)
    int nring = 2 * (W + 2) + 2 * H;
    for (int q = tid; q < nring; q += FNT) {
        int lx, ly;
        if (q < W + 2) { lx = q - 1; ly = -1; }
        else if (q < 2 * (W + 2)) { lx = q - (W + 2) - 1; ly = H; }
        else if (q < 2 * (W + 2) + H) { lx = -1; ly = q - 2 * (W + 2); }
        else { lx = W; ly = q - 2 * (W + 2) - H; }
        int X = x0 + lx, Y = y0 + ly;
        X = X < 0 ? X + L.nx : (X >= L.nx ? X - L.nx : X);
        Y = Y < 0 ? Y + L.ny : (Y >= L.ny ? Y - L.ny : Y);
        long long s = (long long)X + (long long)L.nx * Y + zoff;
        C r0, r1;
        int nd;
        if (L.mask[s]) {
            r0 = psi[2 * s];
            r1 = psi[2 * s + 1];
            nd = L.owner[s];
        } else if (L.dense_psi) {
            r0 = psi[2 * s];
            r1 = psi[2 * s + 1];
            nd = ND_FLUID;
        } else {
            r0 = 0;
            r1 = 0;
#pragma unroll
            for (int i = 0; i < Q; i++) {
                r0 += ld_pop(f + pop_index(i, s, L.pstride), pop_shift<S, C>(L, 0, i));
                r1 += ld_pop(f + pop_index(Q + i, s, L.pstride), pop_shift<S, C>(L, 1, i));
            }
            nd = ND_FLUID;
        }
        sh.psi[slot][0][ly + 1][lx + 1] = r0;
        sh.psi[slot][1][ly + 1][lx + 1] = r1;
        sh.nd[slot][ly + 1][lx + 1] = nd;
    }
    return loaded;
}

// Links of a site that bounce back (Eqs. 9, 17, 18): their neighbour is a
// particle node or lies beyond a wall.  p0 is the particle of the first
// particle link, pm the links into p0; a site next to two particles (multi)
// rewrites the links into the second one after the main store loop.
struct LinkInfo {
    unsigned bb, pm;
    int p0;
    bool multi;
};

template <typename SH>
__device__ __forceinline__ LinkInfo link_info(const SH& sh, const int (&sl)[3], int tx, int ty, bool solid) {
    LinkInfo li = {0u, 0u, -1, false};
#pragma unroll
    for (int i = 1; i < Q; i++) {
        int nd = sh.nd[sl[cz(i) + 1]][ty + 1 + cy(i)][tx + 1 + cx(i)];
        li.bb |= (unsigned)(nd != ND_FLUID) << i;
        if (nd >= 0) {
            li.multi |= li.p0 >= 0 && nd != li.p0;
            li.p0 = li.p0 < 0 ? nd : li.p0;
            li.pm |= (unsigned)(nd == li.p0) << i;
        }
    }
    if (solid) li = LinkInfo{0u, 0u, li.p0, false};
    return li;
}

// Collide and push the own site of plane z (slots: below, here, above); the
// populations are in the stage, rho and j in `m`; `li` and `pref` are the
// site's links and the record of particle li.p0 (any record when li.pm = 0:
// U0 is then unused).  A particle node of the tile (`solid`) runs the same
// instructions and stores the rest equilibrium w_i rho0^k into its own slots
// of f(t+1) instead: no link pushes into a particle node, so without this its
// slots would stay unwritten and the 32-byte sectors they share with fluid
// nodes along every row through a particle would be written only in part
// (each then costs a DRAM read to merge); sharing the store instructions with
// the fluid lanes of the warp keeps the number of store requests that of a
// fluid warp.  The values are never read: a node released by a particle is
// refilled (Eq. 25) before it streams.  (Its arithmetic uses finite moments:
// the populations of a particle node are the stored rest equilibrium.)
// Nearly every warp holds a bounce-back site, so the store of each link
// selects its destination (the neighbour's slot i, or the own slot opp(i)
// with the wall-velocity term) instead of branching.
template <int PREC, bool SR, typename SH, typename PopFn>
__device__ __forceinline__ void collide_site(const Lattice& L, SH& sh, const int (&sl)[3], int x, int y, int z,
                                             int ty, const OwnSite<PREC>& m, bool solid, PopFn pop,
                                             const LinkInfo& li, const ParticleRef<typename Prec<PREC>::C>& pref,
                                             int& pforce, typename Prec<PREC>::C (&Fp)[3],
                                             typename Prec<PREC>::C (&Tp)[3]) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    int tx = threadIdx.x;  // (ty: the shared-memory row of the site, less one)
    const unsigned bb = li.bb, pm = li.pm;
    const int p0 = li.p0;
    const bool multi = li.multi;
    // Eq. 11 (repulsive sign) + body force from the shared-memory psi planes
    C sA[3] = {0, 0, 0}, sB[3] = {0, 0, 0};
#pragma unroll
    for (int i = 1; i < Q; i++) {
        int slot = sl[cz(i) + 1];
        C pa = sh.psi[slot][0][ty + 1 + cy(i)][tx + 1 + cx(i)];
        C pb = sh.psi[slot][1][ty + 1 + cy(i)][tx + 1 + cx(i)];
        C w = wgt<C>(i);
        if (cx(i)) { sA[0] += C(cx(i)) * w * pa; sB[0] += C(cx(i)) * w * pb; }
        if (cy(i)) { sA[1] += C(cy(i)) * w * pa; sB[1] += C(cy(i)) * w * pb; }
        if (cz(i)) { sA[2] += C(cz(i)) * w * pa; sB[2] += C(cz(i)) * w * pb; }
    }
    C F[2][3];
    C G = prm<C>(L.P.G, L.PF.G);
#pragma unroll
    for (int d = 0; d < 3; d++) {
        C g = prm<C>(L.P.body_force[d], L.PF.body_force[d]);
        F[0][d] = -G * m.rho[0] * sB[d] + m.rho[0] * g;
        F[1][d] = -G * m.rho[1] * sA[d] + m.rho[1] * g;
    }
    if (!solid && !(m.rho[0] >= C(0) && m.rho[1] >= C(0) && m.rho[0] < C(1e30) && m.rho[1] < C(1e30)))
        atomicOr(L.flags, FLAG_NONFINITE);
    C u[3], om;
    mixture<C>(L, m.rho, m.j, u, om);
    C us[2][3];
    C tiny = sizeof(C) == 8 ? C(1e-300) : C(1e-30);
#pragma unroll
    for (int k = 0; k < 2; k++) {
        C ir = m.rho[k] > tiny ? C(1) / m.rho[k] : C(0);
#pragma unroll
        for (int d = 0; d < 3; d++) us[k][d] = u[d] + F[k][d] * ir;
    }
    C uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    C uus[2] = {us[0][0] * us[0][0] + us[0][1] * us[0][1] + us[0][2] * us[0][2],
                us[1][0] * us[1][0] + us[1][1] * us[1][1] + us[1][2] * us[1][2]};
    C one_m_om = C(1) - om;
    // 3 w_c rho^k per weight class c (1 axis, 2 diagonal): the wall term of
    // the bounce-back (Eqs. 9, 17) is 3 w_c rho^k (-2 c_i.u_w)
    C B[2][3];
#pragma unroll
    for (int k = 0; k < 2; k++)
#pragma unroll
        for (int c = 0; c < 3; c++) B[k][c] = C(3) * (wgt<C>(c == 0 ? 0 : (c == 1 ? 1 : 7)) * m.rho[k]);
    // site-index steps to the neighbours, periodic wrap folded in (32-bit:
    // a lattice holds fewer than 2^31 sites)
    const unsigned ps = (unsigned)L.pstride;
    const int nx = L.nx, nxy = L.nx * L.ny;
    const unsigned s = (unsigned)x + (unsigned)nx * ((unsigned)y + (unsigned)L.ny * (unsigned)z);
    const int dxp = x == nx - 1 ? 1 - nx : 1, dxm = x == 0 ? nx - 1 : -1;
    const int dyp = y == L.ny - 1 ? nx - nxy : nx, dym = y == 0 ? nxy - nx : -nx;
    const int dzp = z == L.nz - 1 ? nxy - (int)L.N : nxy, dzm = z == 0 ? (int)L.N - nxy : -nxy;
    const bool wall_lo = z == 0 && !L.per[2], wall_hi = z == L.nz - 1 && !L.per[2];
    C U0[3], rel[3];
    particle_u0_of<C>(L, pref, x, y, z, U0, rel);
    // Eq. 19: the momentum a link into p0 hands over, (f*_i + f_ibar(t+1)) c_i
    C Fl[3] = {0, 0, 0};
    // wall velocity of the links leaving through z-1 / z / z+1 (a site next
    // to a wall bounces its wall links on the wall, all others on U0)
    C V[3][3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        V[0][d] = wall_lo ? prm<C>(L.P.wall_u_lo[d], L.PF.wall_u_lo[d]) : U0[d];
        V[1][d] = U0[d];
        V[2][d] = wall_hi ? prm<C>(L.P.wall_u_hi[d], L.PF.wall_u_hi[d]) : U0[d];
    }
    // destinations as 32-bit pair offsets from the base of the plane pair
    // (2j-1, 2j): plane 2j adds ps; a pair of plane i is SKEW + site - c_ix
    // (pair_index); sites < 2^31 and ps < 2^31 keep them in range
    S* const fn = (S*)L.f_nxt;
    auto pair_at = [&](int plane, unsigned off) { return fn + 2 * ((unsigned long long)ps * (unsigned)plane + off); };
    // FP16 with stochastic rounding (SR, a separate instantiation): the
    // rounding bits of this site; both components of a link are stored by
    // one call
    unsigned rs = 0;
    if constexpr (SR) rs = sr_start(s, L.sr_key);
    auto put2 = [&](S* p, C va, C vb, C sa, C sb) {
        if constexpr (SR) {
            st_pair_sr(p, va, vb, sa, sb, sr_next2(rs));
        } else {
            st_pair(p, va, vb, sa, sb);
        }
    };
#pragma unroll
    for (int i = 0; i < Q; i++) {
        C fs[2];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            fs[k] = one_m_om * (ld_pop(pop(k * Q + i), pop_shift<S, C>(L, k, i)) -
                                feq<C>(i, m.rho[k], u[0], u[1], u[2], uu)) +
                    feq<C>(i, m.rho[k], us[k][0], us[k][1], us[k][2], uus[k]);
        }
        if (i == 0) {
            put2(pair_at(0, (unsigned)SKEW + s), solid ? wgt<C>(0) * prm<C>(L.P.rho0[0], L.PF.rho0[0]) : fs[0],
                 solid ? wgt<C>(0) * prm<C>(L.P.rho0[1], L.PF.rho0[1]) : fs[1], pop_shift<S, C>(L, 0, 0),
                 pop_shift<S, C>(L, 1, 0));
            continue;
        }
        const int lo = (i & 1) ? i : i - 1;  // first plane of the pair
        const bool b = (bb >> i) & 1u;
        const unsigned q = solid ? s
                                 : s + (unsigned)((cx(i) > 0 ? dxp : (cx(i) < 0 ? dxm : 0)) +
                                                  (cy(i) > 0 ? dyp : (cy(i) < 0 ? dym : 0)) +
                                                  (cz(i) > 0 ? dzp : (cz(i) < 0 ? dzm : 0)));
        // push: the destination's element of plane i, SKEW + q - c_ix (at the
        // source's x); bounce-back: the own element of plane opp(i),
        // SKEW + s + c_ix
        const unsigned off = b ? (unsigned)(SKEW + cx(i)) + s + (opp(i) == lo ? 0u : ps)
                               : (unsigned)(SKEW - cx(i)) + q + (i == lo ? 0u : ps);
        const int zs = cz(i) + 1;
        C cw = C(cx(i)) * V[zs][0] + C(cy(i)) * V[zs][1] + C(cz(i)) * V[zs][2];
        cw = b ? C(-2) * cw : C(0);  // f_ibar = f*_i - 6 w_i rho c_i.u_w (Eq. 17)
        const int c = i <= 6 ? 1 : 2;
        C fb[2];
#pragma unroll
        for (int k = 0; k < 2; k++) fb[k] = fs[k] + B[k][c] * cw;
        put2(pair_at(lo, off), solid ? wgt<C>(i) * prm<C>(L.P.rho0[0], L.PF.rho0[0]) : fb[0],
             solid ? wgt<C>(i) * prm<C>(L.P.rho0[1], L.PF.rho0[1]) : fb[1], pop_shift<S, C>(L, 0, i),
             pop_shift<S, C>(L, 1, i));
        C fl = fs[0] + fb[0] + fs[1] + fb[1];
        fl = (pm >> i) & 1u ? fl : C(0);
        if (cx(i)) Fl[0] += C(cx(i)) * fl;
        if (cy(i)) Fl[1] += C(cy(i)) * fl;
        if (cz(i)) Fl[2] += C(cz(i)) * fl;
    }
    // Eq. 23 with r_w - r_p = (x - r_p) + c_i/2: the c_i/2 part is parallel
    // to the link force and drops out of the torque
    pforce = pm ? p0 : -1;
#pragma unroll
    for (int d = 0; d < 3; d++) Fp[d] = Fl[d];
    Tp[0] = rel[1] * Fl[2] - rel[2] * Fl[1];
    Tp[1] = rel[2] * Fl[0] - rel[0] * Fl[2];
    Tp[2] = rel[0] * Fl[1] - rel[1] * Fl[0];
    // open z faces of the pressure (Eq. 10) or equilibrium kind, and velocity
    // faces with extrapolated densities: rewrite the populations the face
    // sends in (the loop above stored the wall rule)
    const int face = wall_lo ? 0 : (wall_hi ? 1 : -1);
    const int ftype = face >= 0 ? L.P.open[face] : 0;
    const bool fext = L.P.open_extrap && (ftype == 1 || ftype == 2);
    if (face >= 0 && !solid && (ftype == 1 || ftype == 3 || fext)) {
        // u_w of a pressure face: the velocity of this node, or the
        // extrapolated one (k_face_values), which also holds rho_w^k of a
        // velocity face
        const C* fv = (const C*)L.face + 5 * ((long long)face * L.nx * L.ny + x + (long long)L.nx * y);
        C ue[3];
#pragma unroll
        for (int d = 0; d < 3; d++) ue[d] = fext ? fv[2 + d] : u[d];
        const C ueu = ue[0] * ue[0] + ue[1] * ue[1] + ue[2] * ue[2];
        const C* uw = V[face == 0 ? 0 : 2];
        const C uwu = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
#pragma unroll 1
        for (int i = 1; i < Q; i++) {
            if (cz(i) != (face == 0 ? -1 : 1)) continue;
            C fb[2];
            for (int k = 0; k < 2; k++) {
                const C rw = C(L.P.open_rho[face][k]);
                if (ftype != 3) {
                    const C fsk = one_m_om * (ld_pop(pop(k * Q + i), pop_shift<S, C>(L, k, i)) -
                                              feq<C>(i, m.rho[k], u[0], u[1], u[2], uu)) +
                                  feq<C>(i, m.rho[k], us[k][0], us[k][1], us[k][2], uus[k]);
                    if (ftype == 1) {
                        // -f*_i + 2 w_i rho_w (1 + 9/2 (c_i.u_w)^2 - 3/2 u_w.u_w)
                        const C cuw = C(cx(i)) * ue[0] + C(cy(i)) * ue[1] + C(cz(i)) * ue[2];
                        fb[k] = -fsk + C(2) * wgt<C>(i) * rw * (C(1) + C(4.5) * cuw * cuw - C(1.5) * ueu);
                    } else {
                        // Eq. 9 with the extrapolated rho_w^k: f*_i - 6 w_i rho_w c_i.u_w
                        const C cw = C(cx(i)) * uw[0] + C(cy(i)) * uw[1] + C(cz(i)) * uw[2];
                        fb[k] = fsk - C(6) * (wgt<C>(i) * fv[k]) * cw;
                    }
                } else {
                    fb[k] = feq<C>(opp(i), rw, uw[0], uw[1], uw[2], uwu);
                }
            }
            const unsigned own = (unsigned)(SKEW + cx(i)) + s;  // pair of s in plane opp(i)
            put2(pair_at(opp(i), own), fb[0], fb[1], pop_shift<S, C>(L, 0, opp(i)), pop_shift<S, C>(L, 1, opp(i)));
        }
    }
    if (multi) {
#pragma unroll 1
        for (int i = 1; i < Q; i++) {
            int a = cz(i) < 0 ? sl[0] : (cz(i) > 0 ? sl[2] : sl[1]);
            int nd = sh.nd[a][ty + 1 + cy(i)][tx + 1 + cx(i)];
            if (nd < 0 || nd == p0) continue;
            C U[3], r2[3];
            particle_u0<C>(L, nd, x, y, z, U, r2);
            C cw = C(cx(i)) * U[0] + C(cy(i)) * U[1] + C(cz(i)) * U[2];
            C fsv[2], fbv[2];
            for (int k = 0; k < 2; k++) {
                fsv[k] = one_m_om * (ld_pop(pop(k * Q + i), pop_shift<S, C>(L, k, i)) -
                                     feq<C>(i, m.rho[k], u[0], u[1], u[2], uu)) +
                         feq<C>(i, m.rho[k], us[k][0], us[k][1], us[k][2], uus[k]);
                fbv[k] = fsv[k] - C(6) * wgt<C>(i) * m.rho[k] * cw;
            }
            const unsigned own = (unsigned)(SKEW + cx(i)) + s;  // pair of s in plane opp(i)
            put2(pair_at(opp(i), own), fbv[0], fbv[1], pop_shift<S, C>(L, 0, i), pop_shift<S, C>(L, 1, i));
            const C fl = fsv[0] + fbv[0] + fsv[1] + fbv[1];
            // the link force into the second particle, added directly
            const C F2[3] = {C(cx(i)) * fl, C(cy(i)) * fl, C(cz(i)) * fl};
            const C T2[3] = {r2[1] * F2[2] - r2[2] * F2[1], r2[2] * F2[0] - r2[0] * F2[2],
                             r2[0] * F2[1] - r2[1] * F2[0]};
            for (int d = 0; d < 3; d++) {
                acc_add(L, acc_slot(L, ACC_FLIQ, nd, d), F2[d]);
                acc_add(L, acc_slot(L, ACC_TLIQ, nd, d), T2[d]);
            }
        }
    }
}

template <int PREC, bool SR>
__global__ void __launch_bounds__(FNT, (PREC == LB_FP64 ? 1 : 2)) k_fused(Lattice L, int zc) {
    typedef typename Prec<PREC>::C C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FusedShared<PREC>& sh = *reinterpret_cast<FusedShared<PREC>*>(smem_raw);
    int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
    int W = min(FTX, L.nx - x0), H = min(FTY, L.ny - y0);
    int z0 = blockIdx.z * zc, z1 = min(z0 + zc, L.nz);
    int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FTX + tx;
    bool act = tx < W && ty < H;
    OwnSite<PREC> nxt, cur;
    // prologue: plane z0-1 into slot 0, plane z0 into slot 1 (own site staged)
    fill_plane<PREC>(L, sh, 0, z0 - 1, x0, y0, W, H, false, nxt);
    bool have = fill_plane<PREC>(L, sh, 1, z0, x0, y0, W, H, true, nxt);
    // the populations themselves are needed again for the collision
    if (have)
#pragma unroll
        for (int q = 0; q < 2 * Q; q++) sh.stage[q][tid] = nxt.raw[q];
    cur.rho[0] = nxt.rho[0]; cur.rho[1] = nxt.rho[1];
#pragma unroll
    for (int d = 0; d < 3; d++) { cur.j[0][d] = nxt.j[0][d]; cur.j[1][d] = nxt.j[1][d]; }
    int lo = 0, mid = 1, hi = 2;
    for (int z = z0; z < z1; z++) {
        bool more = z + 1 < z1;
        bool have_n = fill_plane<PREC>(L, sh, hi, z + 1, x0, y0, W, H, more, nxt);
        __syncthreads();
        int pf = -1;
        C Fp[3] = {0, 0, 0}, Tp[3] = {0, 0, 0};
        if (act) {
            int sl[3] = {lo, mid, hi};
            const bool solid = sh.nd[mid][ty + 1][tx + 1] != ND_FLUID;
            const LinkInfo li = link_info(sh, sl, tx, ty, solid);
            // (particle 0 stands in when no link reaches a particle: its
            // record exists whenever the lattice has room for particles)
            const ParticleRef<C> pref = particle_load<C>(L, li.p0 >= 0 ? li.p0 : 0);
            collide_site<PREC, SR>(L, sh, sl, x0 + tx, y0 + ty, z, ty, cur, solid,
                                     [&](int q) { return &sh.stage[q][tid]; }, li, pref, pf, Fp, Tp);
        }
        commit_link_forces<C>(L, pf, Fp, Tp);
        __syncthreads();
        if (have_n)
#pragma unroll
            for (int q = 0; q < 2 * Q; q++) sh.stage[q][tid] = nxt.raw[q];
        cur.rho[0] = nxt.rho[0]; cur.rho[1] = nxt.rho[1];
#pragma unroll
        for (int d = 0; d < 3; d++) { cur.j[0][d] = nxt.j[0][d]; cur.j[1][d] = nxt.j[1][d]; }
        int t = lo; lo = mid; mid = hi; hi = t;
    }
}


// ------------------------------------------ copy-pipelined fused step
// The fused step for a lattice with particles at tau != 1 (tau = 1: the
// lean momentum kernel below), where a full density pass
// (k_density) and the virtual densities (Eq. 20) have filled psi before the
// step: the halo of the Shan-Chen sum then needs no populations, and the
// block streams each plane through shared memory with asynchronous copies
// (cp.async, 16-byte chunks of the tile rows for the populations, 4/8-byte
// copies for psi^k and the owner map of tile + ring), issued one plane ahead
// so that the copies of plane z+1 and of the psi plane z+2 are in flight while
// plane z collides.  One barrier per plane; the population stage is double
// buffered.  Completion is the copy unit's own wait (cp.async.wait_all),
// not a spin.

constexpr int ASYNC_TY = 8;  // tile rows of the copy-pipelined kernel

template <int PREC, int TY>
struct AsyncShared {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    static constexpr int NSLOT = 4;  // psi planes held: z-1, z, z+1 and the one in flight
    // one 16-byte chunk of pairs beyond the tile on each side of a row: the
    // own pair of a site in plane i sits c_ix off its column (pair_index)
    static constexpr int EPC = 16 / (int)sizeof(S);  // elements per chunk
    static constexpr int MS = EPC / 2;               // sites per chunk
    static constexpr int SW = 2 * (FTX + 2 * MS);    // elements of a staged row
    S stage[2][Q][TY][SW];
    C psi[NSLOT][2][TY + 2][RW];
    int nd[NSLOT][TY + 2][RW];
};

// nx (and so every tile width) must be a multiple of this for the 16-byte
// population chunks of a precision
template <int PREC>
constexpr int async_x_multiple() {
    return 16 / (int)sizeof(typename Prec<PREC>::S) < 4 ? 4 : 16 / (int)sizeof(typename Prec<PREC>::S);
}

template <int PREC, int TY, bool SR>
__global__ void __launch_bounds__(FTX* TY, (PREC == LB_FP64 ? 1 : 16 / TY)) k_fused_async(Lattice L, int zc) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    typedef AsyncShared<PREC, TY> SH;
    typedef S E;
    constexpr int NT = FTX * TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SH& sh = *reinterpret_cast<SH*>(smem_raw);
    const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * TY;
    const int W = min(FTX, L.nx - x0), H = min(TY, L.ny - y0);
    const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, L.nz);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FTX + tx;
    const bool act = tx < W && ty < H;
    const long long nxy = (long long)L.nx * L.ny;
    const C* psig = (const C*)L.psi;
    auto slot_of = [&](int p) { return (p - z0 + 1) % SH::NSLOT; };
    // fixed per thread: its own tile position and, for the first 2(W+2) + 2H
    // threads, one position of the ring (periodic images at the edges)
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
    // psi^k and node codes of plane p (tile + ring) into its slot
    auto issue_psi = [&](int p) {
        int slot = slot_of(p);
        if ((p < 0 || p >= L.nz) && !L.per[2]) {
            const C* pw = (const C*)L.psi_wall + 2 * (p < 0 ? 0 : nxy);
            if (act) {
                sh.psi[slot][0][ty + 1][tx + 1] = pw[2 * own_xy];
                sh.psi[slot][1][ty + 1][tx + 1] = pw[2 * own_xy + 1];
                sh.nd[slot][ty + 1][tx + 1] = ND_WALL;
            }
            if (has_ring) {
                sh.psi[slot][0][rly + 1][rlx + 1] = pw[2 * ring_xy];
                sh.psi[slot][1][rly + 1][rlx + 1] = pw[2 * ring_xy + 1];
                sh.nd[slot][rly + 1][rlx + 1] = ND_WALL;
            }
            return;
        }
        int Z = p < 0 ? p + L.nz : (p >= L.nz ? p - L.nz : p);
        const long long zoff = nxy * Z;
        // the owner map is the node code: -1 on fluid nodes
        auto put = [&](int ly, int lx, long long g) {
            cp_async_4(&sh.nd[slot][ly][lx], L.owner + g);
            if (sizeof(C) == 8) {
                cp_async_8(&sh.psi[slot][0][ly][lx], psig + 2 * g);
                cp_async_8(&sh.psi[slot][1][ly][lx], psig + 2 * g + 1);
            } else {
                cp_async_4(&sh.psi[slot][0][ly][lx], psig + 2 * g);
                cp_async_4(&sh.psi[slot][1][ly][lx], psig + 2 * g + 1);
            }
        };
        if (act) put(ty + 1, tx + 1, zoff + own_xy);
        if (has_ring) put(rly + 1, rlx + 1, zoff + ring_xy);
    };
    // the 19 population rows (component pairs) of the tile of plane p into
    // stage buffer b: warp ty copies its row, pairs SKEW + s(x0) - MS ..
    // + FTX + MS of every plane (aligned: x0 and nx are multiples of MS), in
    // 16-byte chunks
    constexpr int EPC = SH::EPC, MS = SH::MS;
    constexpr int WCH = SH::SW / EPC;  // chunks per row
    const long long row_site = (long long)x0 + (long long)L.nx * (y0 + ty);
    auto issue_pops = [&](int p, int b) {
        if (ty >= H) return;
        const E* base = (const E*)L.f_cur + 2 * ((SKEW - MS) + row_site + nxy * p);
        for (int c = tx; c < Q * WCH; c += FTX) {
            const int q = c / WCH, ch = c - q * WCH;
            cp_async_16(&sh.stage[b][q][ty][ch * EPC], base + 2 * (long long)q * L.pstride + ch * EPC);
        }
    };
    for (int p = z0 - 1; p < z0 + 2; p++)
        if (p <= z1) issue_psi(p);
    issue_pops(z0, 0);
    cp_async_commit();
    for (int z = z0; z < z1; z++) {
        cp_async_wait_all();
        __syncthreads();
        const int b = (z - z0) & 1;
        if (z + 1 < z1) issue_pops(z + 1, b ^ 1);
        if (z + 2 <= z1) issue_psi(z + 2);
        cp_async_commit();
        int pf = -1;
        C Fp[3] = {0, 0, 0}, Tp[3] = {0, 0, 0};
        if (act) {
            const int mid = slot_of(z);
            OwnSite<PREC> m;
#pragma unroll
            for (int k = 0; k < 2; k++) {
                C r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
                for (int i = 0; i < Q; i++) {
                    C v = ld_pop(&sh.stage[b][i][ty][2 * (MS + tx - cx(i)) + k], pop_shift<S, C>(L, k, i));
                    r += v;
                    if (cx(i) > 0) jx += v; else if (cx(i) < 0) jx -= v;
                    if (cy(i) > 0) jy += v; else if (cy(i) < 0) jy -= v;
                    if (cz(i) > 0) jz += v; else if (cz(i) < 0) jz -= v;
                }
                m.rho[k] = r;
                m.j[k][0] = jx; m.j[k][1] = jy; m.j[k][2] = jz;
            }
            int sl[3] = {slot_of(z - 1), mid, slot_of(z + 1)};
            const bool solid = sh.nd[mid][ty + 1][tx + 1] != ND_FLUID;
            const LinkInfo li = link_info(sh, sl, tx, ty, solid);
            const ParticleRef<C> pref = particle_load<C>(L, li.p0 >= 0 ? li.p0 : 0);
            collide_site<PREC, SR>(L, sh, sl, x0 + tx, y0 + ty, z, ty, m, solid,
                                     [&](int q) { return &sh.stage[b][q % Q][ty][2 * (MS + tx - cx(q % Q)) + q / Q]; },
                                     li, pref,
                                     pf, Fp, Tp);
        }
        commit_link_forces<C>(L, pf, Fp, Tp);
    }
    cp_async_wait_all();
}

static int z_chunks(const Lattice& L, int tiles, int per_sm, int zmin);

constexpr int WNSLOT = 5;  // psi planes a lean warp holds: z-1 .. z+3
constexpr int WPB = 4;     // warps (rows) per block of the lean kernel

// ------------------------------------------------------- lean momentum kernel
// At omega = 1 (tau^A = tau^B = 1), with or without particles, and the class of
// every link kept with the node map (nb, NB_*), this kernel collides every
// site from its moments (Eq. 16 at omega = 1, with the force of Eq. 11) and
// pushes its links (Eq. 3) with no per-link decisions beyond a predicate:
//   - a fluid site pushes all 19 links; a link into a particle node lands in
//     that node's storage, which is never read as populations (the density
//     pass gives particle nodes zero moments, and a node released by a
//     particle is refilled (Eq. 25) before it streams);
//   - a particle node collides on the rest density rho0^k (finite values)
//     and pushes its links except those into fluid sites, whose elements
//     the fluid sites' bounce-back fills;
//   - a fluid site with links into particle nodes also writes, for each of
//     them, f_ibar(x, t+1) = f*_i - 6 w_i rho^k c_i.u_w (Eqs. 17, 18) into its
//     own element of plane opp(i), with f*_i still in registers, and sums the
//     momentum the links hand over (Eqs. 19, 22, 23); the branch is taken per
//     link only when some lane of the warp has that link;
//   - a link across a wall plane wraps to the opposite face, where
//     k_wall_bounce applies the face rules.
// So every element of f(t+1) is written exactly once, by one store of a
// warp-wide instruction (no sector is left partly written), and the per-site
// code stays short: the fused march with per-link classification in shared
// memory spent most of its issue slots there.
template <int PREC>
struct alignas(16) LeanShared {
    typedef typename Prec<PREC>::C C;
    C pad_[2];                   // puts column 1 (the tile's first site) on a 16-byte boundary
    C psi[WNSLOT][3][RW][2];     // psi^A, psi^B side by side: one shared load per neighbour
    alignas(16) C j[2][3][FTX];  // j^A + j^B; 16-byte copies land here
};
static_assert(offsetof(LeanShared<LB_FP32>, j) % 16 == 0 && sizeof(LeanShared<LB_FP32>) % 16 == 0, "alignment");
static_assert(offsetof(LeanShared<LB_FP64>, j) % 16 == 0 && sizeof(LeanShared<LB_FP64>) % 16 == 0, "alignment");
// 16-byte chunks land on column 1 + k SPC of a row
static_assert((offsetof(LeanShared<LB_FP32>, psi) + 2 * sizeof(float)) % 16 == 0 && (RW * 2 * sizeof(float)) % 16 == 0,
              "alignment");
static_assert((offsetof(LeanShared<LB_FP64>, psi) + 2 * sizeof(double)) % 16 == 0, "alignment");

// The link forces and torques of one lane summed over the planes of its
// march while they go to one particle p, added to p's fixed-point sums
// (Eqs. 22, 23) when the particle changes and at the end of the march: a
// particle spans several planes, so this saves most of the atomics.  The
// order of the FP additions is fixed by the march, so the sums are the same
// bits on every run.
template <typename C>
struct LinkSum {
    int p;
    C F[3], T[3];
};

// Collide the site (x, y, z) of the warp's row and push its 19 links
// (slots: psi planes z-1, z, z+1; b: the momentum buffer of plane z).
template <int PREC, bool SR, bool NEAR>
__device__ __forceinline__ void lean_site(const Lattice& L, const LeanShared<PREC>& sh, const int (&sl)[3], int x,
                                          int y, int z, int b, uint32_t nbc,
                                          LinkSum<typename Prec<PREC>::C>& ls) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    const int tx = threadIdx.x;
    const bool solid = nbc & NB_SOLID;
    C rho[2];
#pragma unroll
    for (int k = 0; k < 2; k++) rho[k] = solid ? prm<C>(L.P.rho0[k], L.PF.rho0[k]) : sh.psi[sl[1]][1][tx + 1][k];
    // Eq. 11 (repulsive sign) + body force from the staged psi planes
    C sA[3] = {0, 0, 0}, sB[3] = {0, 0, 0};
#pragma unroll
    for (int i = 1; i < Q; i++) {
        const int slot = sl[cz(i) + 1];
        const C pa = sh.psi[slot][1 + cy(i)][tx + 1 + cx(i)][0];
        const C pb = sh.psi[slot][1 + cy(i)][tx + 1 + cx(i)][1];
        const C w = wgt<C>(i);
        if (cx(i)) { sA[0] += C(cx(i)) * w * pa; sB[0] += C(cx(i)) * w * pb; }
        if (cy(i)) { sA[1] += C(cy(i)) * w * pa; sB[1] += C(cy(i)) * w * pb; }
        if (cz(i)) { sA[2] += C(cz(i)) * w * pa; sB[2] += C(cz(i)) * w * pb; }
    }
    const C G = prm<C>(L.P.G, L.PF.G);
    // Eq. 14 at tau_A = tau_B: u = (j^A + j^B) / (rho^A + rho^B) (j = 0 on
    // particle nodes)
    C us[2][3], u[3];
    {
        const C ir = C(1) / (rho[0] + rho[1]);
#pragma unroll
        for (int d = 0; d < 3; d++) u[d] = sh.j[b][d][tx] * ir;
    }
    const C tiny = sizeof(C) == 8 ? C(1e-300) : C(1e-30);
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const C ir = rho[k] > tiny ? C(1) / rho[k] : C(0);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const C g = prm<C>(L.P.body_force[d], L.PF.body_force[d]);
            const C F = -G * rho[k] * (k == 0 ? sB[d] : sA[d]) + rho[k] * g;
            us[k][d] = u[d] + F * ir;  // Eq. 16: the shifted velocity
        }
    }
    // Eq. 5 factored per weight class c (0 rest, 1 axis, 2 diagonal):
    // f^eq_i = A_c + c_i.us (B_c + H_c c_i.us), A_c = w_c rho (1 - 3/2 us.us),
    // B_c = 3 w_c rho, H_c = 9/2 w_c rho
    C A[2][3], B[2][3], H[2][3];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const C uus = us[k][0] * us[k][0] + us[k][1] * us[k][1] + us[k][2] * us[k][2];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const C wr = wgt<C>(c == 0 ? 0 : (c == 1 ? 1 : 7)) * rho[k];
            A[k][c] = wr * (C(1) - C(1.5) * uus);
            B[k][c] = C(3) * wr;
            H[k][c] = C(4.5) * wr;
        }
    }
    // destinations as pair offsets from the site's pair of plane 0 (pA): the
    // pair of plane i at site q is i ps + SKEW + q - c_ix, so the shift by
    // c_ix cancels and only the periodic wrap in x is left.  NEAR: the
    // offsets fit in 32 bits ((Q - 1) ps + N < 2^31, checked by the
    // launcher), so an address is one wide multiply-add from the site's
    // pointer
    typedef typename std::conditional<NEAR, int, long long>::type Off;
    const Off ps = (Off)L.pstride;
    const int nx = L.nx, nxy = L.nx * L.ny;
    const unsigned s = (unsigned)x + (unsigned)nx * ((unsigned)y + (unsigned)L.ny * (unsigned)z);
    const int wxp = x == nx - 1 ? -nx : 0, wxm = x == 0 ? nx : 0;
    const int dyp = y == L.ny - 1 ? nx - nxy : nx, dym = y == 0 ? nxy - nx : -nx;
    const int dzp = z == L.nz - 1 ? nxy - (int)L.N : nxy, dzm = z == 0 ? (int)L.N - nxy : -nxy;
    // site-index step to the neighbour along a link known at run time
    auto step_of = [&](int i) {
        const int a = rc(0, i), bb_ = rc(1, i), c = rc(2, i);
        return (unsigned)((a > 0 ? 1 + wxp : (a < 0 ? wxm - 1 : 0)) + (bb_ > 0 ? dyp : (bb_ < 0 ? dym : 0)) +
                          (c > 0 ? dzp : (c < 0 ? dzm : 0)));
    };
    // bounce-back links; a site next to two particles takes the general
    // path after the loop
    const unsigned bb = solid ? 0u : (nbc & NB_LINKS);
    const unsigned bbi = (nbc & NB_MULTI) ? 0u : bb;
    const unsigned wbb = __reduce_or_sync(__activemask(), bbi);  // the links any lane of the warp bounces
    // the particle of the bounce-back links and u_w = v_p + omega_p x (x - r_p)
    C U0[3] = {0, 0, 0}, rel[3] = {0, 0, 0};
    int p0 = -1;
    if (bbi) {
        p0 = L.owner[s + step_of(__ffs(bbi) - 1)];
        particle_u0_of<C>(L, particle_load<C>(L, p0), x, y, z, U0, rel);
    }
    C Fl[3] = {0, 0, 0};  // Eq. 19 summed over the links: (f*_i + f_ibar(t+1)) c_i
    S* const pA = (S*)L.f_nxt + 2 * (SKEW + (long long)s);
    // the rounding bits of the site's stores, in store order (the bounce-back
    // stores of a link follow its push when the warp takes that branch)
    unsigned rs = 0;
    if constexpr (SR) rs = sr_start(s, L.sr_key);
    auto put2 = [&](S* p, C va, C vb, C sa, C sb, bool on, unsigned& st) {
        if constexpr (SR) {
            st_pair_sr_if(p, va, vb, sa, sb, sr_next2(st), on);
        } else {
            st_pair_if(p, va, vb, sa, sb, on);
        }
    };
    put2(pA, A[0][0], A[1][0], pop_shift<S, C>(L, 0, 0), pop_shift<S, C>(L, 1, 0), true, rs);
#pragma unroll
    for (int i = 1; i < Q; i++) {
        const int c = i <= 6 ? 1 : 2;
        C fs[2];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const C cu = C(cx(i)) * us[k][0] + C(cy(i)) * us[k][1] + C(cz(i)) * us[k][2];
            fs[k] = A[k][c] + cu * (B[k][c] + H[k][c] * cu);
        }
        const Off off = (Off)i * ps + (Off)((cx(i) > 0 ? wxp : (cx(i) < 0 ? wxm : 0)) +
                                            (cy(i) > 0 ? dyp : (cy(i) < 0 ? dym : 0)) +
                                            (cz(i) > 0 ? dzp : (cz(i) < 0 ? dzm : 0)));
        // a particle node does not push into a fluid site (whose bounce-back
        // writes that element)
        put2(pA + 2 * (long long)off, fs[0], fs[1], pop_shift<S, C>(L, 0, i), pop_shift<S, C>(L, 1, i),
             !(solid && ((nbc >> i) & 1u)), rs);
        if (wbb & (1u << i)) {
            // Eq. 17 with the wall velocity of Eq. 18: the own element of
            // plane opp(i), opp(i) ps + SKEW + s + c_ix
            const bool on = (bbi >> i) & 1u;
            const C cw = C(-2) * (C(cx(i)) * U0[0] + C(cy(i)) * U0[1] + C(cz(i)) * U0[2]);
            C fb[2];
#pragma unroll
            for (int k = 0; k < 2; k++) fb[k] = fs[k] + B[k][c] * cw;
            const Off ob = (Off)opp(i) * ps + cx(i);
            put2(pA + 2 * (long long)ob, fb[0], fb[1], pop_shift<S, C>(L, 0, opp(i)), pop_shift<S, C>(L, 1, opp(i)), on,
                 rs);
            const C fl = on ? fs[0] + fb[0] + fs[1] + fb[1] : C(0);
            if (cx(i)) Fl[0] += C(cx(i)) * fl;
            if (cy(i)) Fl[1] += C(cy(i)) * fl;
            if (cz(i)) Fl[2] += C(cz(i)) * fl;
        }
    }
    if (bbi) {
        // Eq. 23 with r_w - r_p = (x - r_p) + c_i/2: the c_i/2 part is
        // parallel to the link force and drops out of the torque
        if (ls.p != p0) {
            commit_link_forces<C>(L, ls.p, ls.F, ls.T);
            ls = LinkSum<C>{p0, {0, 0, 0}, {0, 0, 0}};
        }
        ls.F[0] += Fl[0];
        ls.F[1] += Fl[1];
        ls.F[2] += Fl[2];
        ls.T[0] += rel[1] * Fl[2] - rel[2] * Fl[1];
        ls.T[1] += rel[2] * Fl[0] - rel[0] * Fl[2];
        ls.T[2] += rel[0] * Fl[1] - rel[1] * Fl[0];
    }
    if (bb && (nbc & NB_MULTI)) {
        // a site next to two particles: each link with its own particle
        unsigned m = bb;
        while (m) {
            const int i = __ffs(m) - 1;
            m &= m - 1;
            const int p = L.owner[s + step_of(i)];
            C U[3], r2[3];
            particle_u0<C>(L, p, x, y, z, U, r2);
            const int ax = rc(0, i), ay = rc(1, i), az = rc(2, i);
            const int c = i <= 6 ? 1 : 2;
            const C cw = C(-2) * (C(ax) * U[0] + C(ay) * U[1] + C(az) * U[2]);
            C fs[2], fb[2];
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const C Ak = c == 1 ? A[k][1] : A[k][2], Bk = c == 1 ? B[k][1] : B[k][2];
                const C Hk = c == 1 ? H[k][1] : H[k][2];
                const C cu = C(ax) * us[k][0] + C(ay) * us[k][1] + C(az) * us[k][2];
                fs[k] = Ak + cu * (Bk + Hk * cu);
                fb[k] = fs[k] + Bk * cw;
            }
            const int o = opp(i);
            S* f = (S*)L.f_nxt;
            put2(f + pair_index(o, s, L.pstride), fb[0], fb[1],
                 pop_shift<S, C>(L, 0, o), pop_shift<S, C>(L, 1, o), true, rs);
            const C fl = fs[0] + fb[0] + fs[1] + fb[1];
            const C F2[3] = {C(ax) * fl, C(ay) * fl, C(az) * fl};
            const C T2[3] = {r2[1] * F2[2] - r2[2] * F2[1], r2[2] * F2[0] - r2[0] * F2[2],
                             r2[0] * F2[1] - r2[1] * F2[0]};
            commit_link_forces<C>(L, p, F2, T2);
        }
    }
}

// One warp per row of 32 sites marching along z through a chunk of planes,
// staging with cp.async (warps wait only for their own copies) psi^k of the
// rows y-1, y, y+1 with the x ring for planes z-1 .. z+3 and the momentum
// rows of the next plane; a plane beyond a wall stages the wall densities.
template <int PREC, bool SR, bool NEAR>
__global__ void __launch_bounds__(FTX* WPB, (PREC == LB_FP64 ? 1 : (PREC == LB_FP16 ? 4 : 5))) k_lean(Lattice L, int zc) {
    typedef typename Prec<PREC>::C C;
    typedef LeanShared<PREC> SH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SH& sh = reinterpret_cast<SH*>(smem_raw)[threadIdx.y];
    const int tx = threadIdx.x;
    const int x0 = blockIdx.x * FTX, y = blockIdx.y * WPB + threadIdx.y;
    if (y >= L.ny) return;  // the whole warp: no block-wide barrier follows
    const int W = min(FTX, L.nx - x0);
    const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, L.nz);
    const bool act = tx < W;
    const long long nxy = (long long)L.nx * L.ny;
    const C* psig = (const C*)L.psi;
    auto slot_of = [&](int p) { return (p - z0 + 1) % WNSLOT; };
    // the psi pairs of the rows y-1, y, y+1 of a plane, as copies of 16-byte
    // chunks (SPC sites each) of the tile's columns and one pair on each side
    // (the periodic images at the lattice edges): 3 (W / SPC + 2) copies, at
    // most two per lane, fixed for the whole march
    constexpr int SPC = 16 / (2 * (int)sizeof(C));
    constexpr int NR = (3 * (FTX / SPC + 2) + 31) / 32;  // copies per lane: 2 (FP32, FP16), 4 (FP64)
    const int nch = W / SPC, per_row = nch + 2;          // W is a multiple of 4 (nx is)
    int jsm[NR], jxy[NR];
    bool jon[NR], jck[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) {
        const int j = tx + 32 * r, row = j / per_row, e = j - row * per_row;
        jon[r] = j < 3 * per_row;
        jck[r] = e < nch;
        int Y = y + row - 1;
        Y = Y < 0 ? Y + L.ny : (Y >= L.ny ? Y - L.ny : Y);
        int X = e < nch ? x0 + e * SPC : (e == nch ? x0 - 1 : x0 + W);
        X = X < 0 ? X + L.nx : (X >= L.nx ? X - L.nx : X);
        const int col = e < nch ? 1 + e * SPC : (e == nch ? 0 : W + 1);
        jsm[r] = jon[r] ? (row * RW + col) * 2 : 0;  // element of the slot
        jxy[r] = X + L.nx * Y;
    }
    auto issue_psi = [&](int p) {
        const int slot = slot_of(p);
        const bool wall = (p < 0 || p >= L.nz) && !L.per[2];
        const int Z = p < 0 ? p + L.nz : (p >= L.nz ? p - L.nz : p);
        // a plane beyond a wall stages the wall densities (pairs as well)
        const C* base = wall ? (const C*)L.psi_wall + 2 * (p < 0 ? 0 : nxy) : psig + 2 * nxy * Z;
#pragma unroll
        for (int r = 0; r < NR; r++) {
            if (!jon[r]) continue;
            C* dst = &sh.psi[slot][0][0][0] + jsm[r];
            const C* src = base + 2 * (long long)jxy[r];
            if (SPC == 1 || jck[r])
                cp_async_16(dst, src);  // a chunk of the tile's columns (FP64: one pair)
            else
                cp_async_8(dst, src);   // a pair of the ring (FP32 / FP16)
        }
    };
    // momentum rows of plane p: 16-byte chunks, lane -> chunk tx % LPR of
    // rows tx / LPR, tx / LPR + 32 / LPR, ...
    constexpr int EPC = 16 / (int)sizeof(C), LPR = FTX / EPC, RPP = FTX / LPR;
    const int chunk = tx % LPR, row0 = tx / LPR;
    const bool jcopy = chunk * EPC < W;
    auto issue_mom = [&](int p, int b) {
        if (!jcopy) return;
        const char* src = (const char*)L.mom + ((long long)row0 * L.pstride + (long long)(x0 + chunk * EPC) +
                                                (long long)L.nx * y + nxy * p) * (long long)sizeof(C);
        for (int r = row0; r < 3; r += RPP) {
            cp_async_16(&sh.j[b][r][chunk * EPC], src);
            src += (long long)RPP * L.pstride * (long long)sizeof(C);
        }
    };
    for (int p = z0 - 1; p < z0 + 3; p++)
        if (p <= z1) issue_psi(p);
    issue_mom(z0, 0);
    cp_async_commit();
    const int x = x0 + tx;
    const long long srow = act ? (long long)x + (long long)L.nx * y : 0;
    uint32_t nbn = act ? L.nb[srow + nxy * z0] : 0u;
    LinkSum<C> ls = {-1, {0, 0, 0}, {0, 0, 0}};
    for (int z = z0; z < z1; z++) {
        cp_async_wait_all();
        __syncwarp();
        const int b = (z - z0) & 1;
        if (z + 1 < z1) issue_mom(z + 1, b ^ 1);
        if (z + 3 <= z1) issue_psi(z + 3);
        cp_async_commit();
        const uint32_t nbc = nbn;
        if (act && z + 1 < z1) nbn = L.nb[srow + nxy * (z + 1)];
        if (!act) continue;
        const int sl[3] = {slot_of(z - 1), slot_of(z), slot_of(z + 1)};
        lean_site<PREC, SR, NEAR>(L, sh, sl, x, y, z, b, nbc, ls);
    }
    commit_link_forces<C>(L, ls.p, ls.F, ls.T);
    cp_async_wait_all();
}

template <int P, bool SR, bool NEAR>
static int launch_lean_t(const Lattice& L, cudaStream_t st) {
    const size_t smem = sizeof(LeanShared<P>) * WPB;
    const int per_sm = kernel_setup<k_lean<P, SR, NEAR>>(FTX * WPB, smem);
    int tiles = ((L.nx + FTX - 1) / FTX) * ((L.ny + WPB - 1) / WPB);
    int zc = z_chunks(L, tiles, per_sm, 8);
    dim3 grid((L.nx + FTX - 1) / FTX, (L.ny + WPB - 1) / WPB, (L.nz + zc - 1) / zc);
    k_lean<P, SR, NEAR><<<grid, dim3(FTX, WPB), smem, st>>>(L, zc);
    return 1;
}

template <int P, bool SR>
static int launch_lean_n(const Lattice& L, cudaStream_t st) {
    // the element offsets of a site's links from its plane-0 element
    if ((long long)(Q - 1) * L.pstride + L.N + 2 * SKEW < (1LL << 31)) return launch_lean_t<P, SR, true>(L, st);
    return launch_lean_t<P, SR, false>(L, st);
}

// The links across the z faces after the lean push.  The push of the link
// c_i (c_iz = -1) of the bottom site b = (X, Y, 0) wrapped into the element
// of plane i of the top site t = (X + c_ix, Y + c_iy, nz - 1), and the push of
// opp(i) of t into the element of plane opp(i) of b: exactly the two elements
// the face rules rewrite, so one thread per (b, i) reads both and writes both.
// Rules by face type: wall or velocity face, Eq. 9 with the face velocity,
// f_ibar = f*_i - 6 w_i rho^k c_i.u_w; pressure face, Eq. 10,
// f_ibar = -f*_i + 2 w_i rho_w^k (1 + 9/2 (c_i.u)^2 - 3/2 u.u) with u the
// mixture velocity of the node; equilibrium face, f^eq_ibar(rho_w^k, u_w).
// rho^k and j^k of the node come from the density pass.  A particle node on a
// face keeps what it holds.
template <int PREC, bool SR>
__device__ __forceinline__ void face_rule(const Lattice& L, int face, int i, const typename Prec<PREC>::C (&fs)[2],
                                          long long x, unsigned& rs) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    const C* psi = (const C*)L.psi;
    const C* mom = (const C*)L.mom;
    const double* uwd = face == 0 ? L.P.wall_u_lo : L.P.wall_u_hi;
    const float* uwf = face == 0 ? L.PF.wall_u_lo : L.PF.wall_u_hi;
    const C uw[3] = {prm<C>(uwd[0], uwf[0]), prm<C>(uwd[1], uwf[1]), prm<C>(uwd[2], uwf[2])};
    const int type = L.P.open[face];
    // extrapolated face values (k_face_values) of the column of x
    const C* fv = (const C*)L.face + 5 * (face * (long long)L.nx * L.ny + x % ((long long)L.nx * L.ny));
    const bool ext = L.P.open_extrap && (type == 1 || type == 2);
    C rho[2] = {psi[2 * x], psi[2 * x + 1]};
    if (ext && type == 2) {
        rho[0] = fv[0];
        rho[1] = fv[1];
    }
    C fb[2];
    if (type == 1) {
        // Eq. 14 at tau_A = tau_B from the total momentum of the density pass
        C u[3];
        const C ir = C(1) / (rho[0] + rho[1]);
#pragma unroll
        for (int d = 0; d < 3; d++) u[d] = ext ? fv[2 + d] : mom[d * L.pstride + x] * ir;
        const C uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const C cuw = C(cx(i)) * u[0] + C(cy(i)) * u[1] + C(cz(i)) * u[2];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const C rw = C(L.P.open_rho[face][k]);
            fb[k] = -fs[k] + C(2) * wgt<C>(i) * rw * (C(1) + C(4.5) * cuw * cuw - C(1.5) * uu);
        }
    } else if (type == 3) {
        const C uwu = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
#pragma unroll
        for (int k = 0; k < 2; k++) fb[k] = feq<C>(opp(i), C(L.P.open_rho[face][k]), uw[0], uw[1], uw[2], uwu);
    } else {
        const C cw = C(-2) * (C(cx(i)) * uw[0] + C(cy(i)) * uw[1] + C(cz(i)) * uw[2]);
#pragma unroll
        for (int k = 0; k < 2; k++) fb[k] = fs[k] + C(3) * (wgt<C>(i) * rho[k]) * cw;
    }
    S* p = (S*)L.f_nxt + pair_index(opp(i), x, L.pstride);
    if constexpr (SR) {
        st_pair_sr(p, fb[0], fb[1], pop_shift<S, C>(L, 0, opp(i)), pop_shift<S, C>(L, 1, opp(i)), sr_next2(rs));
    } else {
        st_pair(p, fb[0], fb[1], pop_shift<S, C>(L, 0, opp(i)), pop_shift<S, C>(L, 1, opp(i)));
    }
}

template <int PREC, bool SR>
__global__ void k_wall_bounce(Lattice L) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    const int X = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y;
    if (X >= L.nx) return;
    const long long nxy = (long long)L.nx * L.ny;
    const long long sb = (long long)X + (long long)L.nx * Y;
    const bool fb_ = !L.mask[sb];
    const S* f = (const S*)L.f_nxt;
    unsigned rs = 0;
    if constexpr (SR) rs = sr_start((unsigned)sb, L.sr_key ^ 0x2545F491u);
#pragma unroll
    for (int i = 1; i < Q; i++) {
        if (cz(i) != -1) continue;
        int Xt = X + cx(i), Yt = Y + cy(i);
        Xt = Xt < 0 ? Xt + L.nx : (Xt >= L.nx ? Xt - L.nx : Xt);
        Yt = Yt < 0 ? Yt + L.ny : (Yt >= L.ny ? Yt - L.ny : Yt);
        const long long stp = (long long)Xt + (long long)L.nx * Yt + nxy * (L.nz - 1);
        C a[2], c[2];  // f*_i of b, f*_opp(i) of t
#pragma unroll
        for (int k = 0; k < 2; k++) {
            a[k] = ld_pop(f + pop_index(k * Q + i, stp, L.pstride), pop_shift<S, C>(L, k, i));
            c[k] = ld_pop(f + pop_index(k * Q + opp(i), sb, L.pstride), pop_shift<S, C>(L, k, opp(i)));
        }
        if (fb_) face_rule<PREC, SR>(L, 0, i, a, sb, rs);
        if (!L.mask[stp]) face_rule<PREC, SR>(L, 1, opp(i), c, stp, rs);
    }
}

// the stochastic-rounding instantiations exist for the FP16 form only
template <int P>
static int launch_lean(const Lattice& L, cudaStream_t st) {
    if constexpr (P == LB_FP16)
        if (L.sr) return launch_lean_n<P, true>(L, st);
    return launch_lean_n<P, false>(L, st);
}


// rho^k of the fluid nodes in the planes next to the walls, written to psi
template <int PREC>
__global__ void k_wall_plane_density(Lattice L) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= L.nx) return;
    int y = blockIdx.y, z = blockIdx.z == 0 ? 0 : L.nz - 1;
    long long s = (long long)x + (long long)L.nx * ((long long)y + (long long)L.ny * z);
    if (L.mask[s]) return;
    const S* f = (const S*)L.f_cur;
    C* psi = (C*)L.psi;
    C r0 = 0, r1 = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        r0 += ld_pop(f + pop_index(i, s, L.pstride), pop_shift<S, C>(L, 0, i));
        r1 += ld_pop(f + pop_index(Q + i, s, L.pstride), pop_shift<S, C>(L, 1, i));
    }
    psi[2 * s] = r0;
    psi[2 * s + 1] = r1;
}

// rho^A, rho^B and u = sum_k (j^k + F^k/2)/rho into stage [5][N] (FP64)
template <int PREC>
__global__ void k_fields_out(Lattice L, double* __restrict__ stage) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y, z = blockIdx.z;
    if (x >= L.nx) return;
    long long s = (long long)x + (long long)L.nx * ((long long)y + (long long)L.ny * z);
    if (L.mask[s]) {
        for (int c = 0; c < 5; c++) stage[c * L.N + s] = 0.0;
        return;
    }
    SiteNbr n = site_nbr(L, x, y, z);
    C fv[2][Q], rho[2], j[2][3], F[2][3];
    load_site<PREC>(L, (const S*)L.f_cur, s, fv, rho, j);
    sc_force<C>(L, n, rho, F);
    C rt = rho[0] + rho[1];
    stage[s] = rho[0];
    stage[L.N + s] = rho[1];
    for (int d = 0; d < 3; d++)
        stage[(2 + d) * L.N + s] =
            double((j[0][d] + C(0.5) * F[0][d] + j[1][d] + C(0.5) * F[1][d]) / rt);
}

// block partial sums of mass, j and j + F/2 (Neumaier, fixed order)
template <int PREC>
__global__ void __launch_bounds__(256) k_totals_partial(Lattice L) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    NSum acc[8];
    for (int a = 0; a < 8; a++) acc[a].s = acc[a].c = 0.0;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < L.N; s += stride) {
        if (L.mask[s]) continue;
        int x = int(s % L.nx), y = int((s / L.nx) % L.ny), z = int(s / ((long long)L.nx * L.ny));
        SiteNbr n = site_nbr(L, x, y, z);
        C fv[2][Q], rho[2], j[2][3], F[2][3];
        load_site<PREC>(L, (const S*)L.f_cur, s, fv, rho, j);
        sc_force<C>(L, n, rho, F);
        for (int k = 0; k < 2; k++) {
            acc[k].add(double(rho[k]));
            for (int d = 0; d < 3; d++) {
                acc[2 + d].add(double(j[k][d]));
                acc[5 + d].add(double(j[k][d] + C(0.5) * F[k][d]));
            }
        }
    }
    __shared__ double sh[256][2];
    for (int a = 0; a < 8; a++) {
        sh[threadIdx.x][0] = acc[a].s;
        sh[threadIdx.x][1] = acc[a].c;
        __syncthreads();
        if (threadIdx.x == 0) {
            NSum t = {0.0, 0.0};
            for (int q = 0; q < blockDim.x; q++) {
                NSum o = {sh[q][0], sh[q][1]};
                t.merge(o);
            }
            L.red[(blockIdx.x * 8 + a) * 2] = t.s;
            L.red[(blockIdx.x * 8 + a) * 2 + 1] = t.c;
        }
        __syncthreads();
    }
}

__global__ void k_totals_final(Lattice L, int nblocks, double* out) {
    int a = threadIdx.x;
    if (a >= 8) return;
    NSum t = {0.0, 0.0};
    for (int b = 0; b < nblocks; b++) {
        NSum o = {L.red[(b * 8 + a) * 2], L.red[(b * 8 + a) * 2 + 1]};
        t.merge(o);
    }
    out[a] = t.value();
}

template <int PREC>
__global__ void k_pops_out(Lattice L, int k, int i, double* __restrict__ stage) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= L.N) return;
    const S* f = (const S*)L.f_cur;
    stage[s] = double(ld_pop(f + pop_index(k * Q + i, s, L.pstride), pop_shift<S, C>(L, k, i)));
}

__global__ void k_clear_map(Lattice L) {
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= L.N) return;
    L.mask[s] = 0;
    L.owner[s] = -1;
    L.evt[s] = 0;
}

// ------------------------------------------------------------ launchers
static inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

static inline dim3 site_grid(const Lattice& L, int bx) {
    return dim3((unsigned)((L.nx + bx - 1) / bx), (unsigned)L.ny, (unsigned)L.nz);
}
static inline int site_bx(const Lattice& L) { return L.nx >= 128 ? 128 : ((L.nx + 31) / 32) * 32; }

#define DISPATCH(prec, call)                      \
    switch (prec) {                               \
        case LB_FP64: { const int P = LB_FP64; call; break; } \
        case LB_FP32: { const int P = LB_FP32; call; break; } \
        default:      { const int P = LB_FP16; call; break; } \
    }

int launch_init_fields(const Lattice& L, int prec, const double* stage, cudaStream_t st) {
    DISPATCH(prec, (k_init<P><<<nblk(L.N, 256), 256, 0, st>>>(L, stage)));
    return 1;
}

int launch_density(const Lattice& L, int prec, cudaStream_t st) {
    if (L.dense_mom) {
        DISPATCH(prec, (k_density<P, true><<<nblk(L.N, 256), 256, 0, st>>>(L)));
    } else {
        DISPATCH(prec, (k_density<P, false><<<nblk(L.N, 256), 256, 0, st>>>(L)));
    }
    return 1;
}

int launch_wall_bounce(const Lattice& L, int prec, cudaStream_t st) {
    if (L.per[2] || !L.dense_mom) return 0;
    dim3 g((unsigned)((L.nx + 127) / 128), (unsigned)L.ny);
    if (prec == LB_FP16 && L.sr) {
        k_wall_bounce<LB_FP16, true><<<g, 128, 0, st>>>(L);
        return 1;
    }
    DISPATCH(prec, (k_wall_bounce<P, false><<<g, 128, 0, st>>>(L)));
    return 1;
}

int launch_face_values(const Lattice& L, int prec, cudaStream_t st) {
    if (L.per[2] || !L.P.open_extrap) return 0;
    if (L.P.open[0] != 1 && L.P.open[0] != 2 && L.P.open[1] != 1 && L.P.open[1] != 2) return 0;
    dim3 g((unsigned)((L.nx + 127) / 128), (unsigned)L.ny, 2);
    DISPATCH(prec, (k_face_values<P><<<g, 128, 0, st>>>(L)));
    return 1;
}

int launch_wall_psi(const Lattice& L, int prec, cudaStream_t st) {
    if (L.per[2]) return 0;
    dim3 g((unsigned)((L.nx + 127) / 128), (unsigned)L.ny, 2);
    if (prec == LB_FP64) k_wall_psi<double><<<g, 128, 0, st>>>(L);
    else k_wall_psi<float><<<g, 128, 0, st>>>(L);
    return 1;
}

// Number of z chunks for a kernel with `per_sm` resident blocks per SM: the
// grid (tiles x chunks) is close to a whole number of full waves, with
// chunks of at least `zmin` planes.
static int z_chunks(const Lattice& L, int tiles, int per_sm, int zmin) {
    long long R = (long long)device_sms() * per_sm;
    int best = 1;
    double best_eff = 0;
    for (int zc = L.nz; zc >= zmin || zc == L.nz; zc--) {
        long long B = (long long)tiles * ((L.nz + zc - 1) / zc);
        double eff = (double)B / (double)(((B + R - 1) / R) * R);
        if (B >= 4 * R && eff > best_eff + 1e-9) {
            best_eff = eff;
            best = zc;
        }
        if (best_eff >= 0.98) break;
        if (zc <= 1) break;
    }
    if (best_eff == 0) best = zmin < L.nz ? zmin : L.nz;
    return best;
}

template <int P, bool SR>
static int launch_fused_async_t(const Lattice& L, cudaStream_t st) {
    constexpr int TY = ASYNC_TY, NT = FTX * TY;
    typedef AsyncShared<P, TY> SH;
    const size_t smem = sizeof(SH);
    const int per_sm = kernel_setup<k_fused_async<P, TY, SR>>(NT, smem);
    int tiles = ((L.nx + FTX - 1) / FTX) * ((L.ny + TY - 1) / TY);
    int zc = z_chunks(L, tiles, per_sm, 8);
    dim3 grid((L.nx + FTX - 1) / FTX, (L.ny + TY - 1) / TY, (L.nz + zc - 1) / zc);
    k_fused_async<P, TY, SR><<<grid, dim3(FTX, TY), smem, st>>>(L, zc);
    return 1;
}

template <int P>
static int launch_fused_async(const Lattice& L, bool unit, cudaStream_t st) {
    // omega = 1: lb_step has the density pass write the momenta, and the
    // lean kernel collides from them; otherwise the general collision
    if (unit && L.dense_mom) return launch_lean<P>(L, st) + launch_wall_bounce(L, P, st);
    if constexpr (P == LB_FP16)
        if (L.sr) return launch_fused_async_t<P, true>(L, st);
    return launch_fused_async_t<P, false>(L, st);
}

// the plain fused kernel (no particles, tau != 1)
template <int P, bool SR>
static int launch_fused_plain(const Lattice& L, int zc, dim3 grid, cudaStream_t st) {
    const size_t smem = sizeof(FusedShared<P>);
    kernel_setup<k_fused<P, SR>>(FTX * FTY, smem);
    k_fused<P, SR><<<grid, dim3(FTX, FTY), smem, st>>>(L, zc);
    return 1;
}

int launch_fluid_step(const Lattice& L, int prec, cudaStream_t st) {
    // with a full density pass done, the copy-pipelined kernel (its 16-byte
    // population chunks need nx to be a multiple of 16 bytes of elements)
    if (L.dense_psi) {
        bool unit = L.P.tau[0] == 1.0 && L.P.tau[1] == 1.0;
        // the momentum rows are 4- or 8-byte values: any nx (a multiple of 4) fits the chunks
        bool mom = unit && L.dense_mom;
        if (prec == LB_FP32 && (mom || L.nx % async_x_multiple<LB_FP32>() == 0))
            return launch_fused_async<LB_FP32>(L, unit, st);
        if (prec == LB_FP16 && (mom || L.nx % async_x_multiple<LB_FP16>() == 0))
            return launch_fused_async<LB_FP16>(L, unit, st);
        if (prec == LB_FP64 && (mom || L.nx % async_x_multiple<LB_FP64>() == 0))
            return launch_fused_async<LB_FP64>(L, unit, st);
    }
    int tiles = ((L.nx + FTX - 1) / FTX) * ((L.ny + FTY - 1) / FTY);
    // z chunk: enough blocks to fill the GPU a few times over, at least 8 planes
    int zc = (int)((long long)L.nz * tiles / 2400);
    zc = zc < 4 ? 4 : zc;
    zc = zc > L.nz ? L.nz : zc;
    dim3 grid((L.nx + FTX - 1) / FTX, (L.ny + FTY - 1) / FTY, (L.nz + zc - 1) / zc);
    // no particles and tau_A, tau_B not both 1 (at omega = 1 lb_step runs the
    // density pass and the lean kernel, particles or not)
    if (prec == LB_FP16 && L.sr) return launch_fused_plain<LB_FP16, true>(L, zc, grid, st);
    DISPATCH(prec, (launch_fused_plain<P, false>(L, zc, grid, st)));
    return 1;
}

int launch_shell_density(const Lattice& L, int prec, cudaStream_t st) {
    int n = 0;
    if (!L.per[2]) {
        dim3 g((unsigned)((L.nx + 127) / 128), (unsigned)L.ny, 2);
        DISPATCH(prec, (k_wall_plane_density<P><<<g, 128, 0, st>>>(L)));
        n++;
    }
    return n;
}

int launch_fields_out(const Lattice& L, int prec, double* stage, cudaStream_t st) {
    int bx = site_bx(L);
    DISPATCH(prec, (k_fields_out<P><<<site_grid(L, bx), bx, 0, st>>>(L, stage)));
    return 1;
}

int launch_totals(const Lattice& L, int prec, double* out_dev, cudaStream_t st) {
    if (L.ncomp == 1) {
        launch_single_totals_partial(L, prec, st);
    } else {
        DISPATCH(prec, (k_totals_partial<P><<<L.red_blocks, 256, 0, st>>>(L)));
    }
    k_totals_final<<<1, 32, 0, st>>>(L, L.red_blocks, out_dev);
    return 2;
}

int launch_populations_out(const Lattice& L, int prec, int k, int i, double* stage, cudaStream_t st) {
    DISPATCH(prec, (k_pops_out<P><<<nblk(L.N, 256), 256, 0, st>>>(L, k, i, stage)));
    return 1;
}

int launch_clear_map(const Lattice& L, cudaStream_t st) {
    k_clear_map<<<nblk(L.N, 256), 256, 0, st>>>(L);
    return 1;
}

}  // namespace lbgb
