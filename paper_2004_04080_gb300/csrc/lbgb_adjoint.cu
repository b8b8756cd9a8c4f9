// lbgb_adjoint.cu -- reverse mode of the lattice step for fixed particles.
//
// With the particles held fixed (infinite mass, zero velocity) the node map
// is static and the time step is a smooth map f(t) -> f(t+1) of the
// populations with parameters tau_A, tau_B, G, zeta_A, zeta_B.  Its adjoint
// takes lambda(t+1) = dJ/df(t+1) to lambda(t) = dJ/df(t) and accumulates the
// parameter gradients.  The forward quantities of step t are recomputed from
// the stored populations f(t) (the caller keeps sqrt(N) checkpoints and
// re-runs each segment).
//
// An adjoint field is stored as lambda_i(x) = L_i(x) + R(x): 2 x 19 local
// values L and a per-site, per-component scalar R added to every link (the
// density adjoint arriving through the Shan-Chen halo), so the non-local part
// costs 2 values per site instead of 38.  Layout in the compute type:
// [L: 2][19][pstride] then [R: 2][pstride].
//
// Forward map at a fluid site x (Sec. 2.3, Eqs. 5-7, 11, 13-16, with the
// readings of the forward kernels):
//   rho^k = sum f^k_i, j^k = sum f^k_i c_i
//   S^k = sum_i w_i psi^k(x + c_i) c_i,  F^A = -G rho^A S^B + rho^A g (A<->B)
//   u = (om_A j^A + om_B j^B) / (om_A rho^A + om_B rho^B), om_k = 1/tau_k
//   om = 1/(3 nubar + 1/2), 1/nubar = sum_k (rho^k/rho)/nu_k, nu_k = (tau_k - 1/2)/3
//   v^k = u + F^k/rho^k
//   f*^k_i = (1 - om)(f^k_i - E_i(rho^k, u)) + E_i(rho^k, v^k)
//   push to x + c_i, or bounce back (Eqs. 8, 9, 17 with u_w = 0 on particles)
// psi is rho on fluid nodes, the virtual density (Eq. 20) on particle frontier
// nodes and the wall density beyond walls; the link forces of Eq. 19 are
// F_p = sum_links sum_k 2 f*^k_i c_i.
#include "lbgb_internal.cuh"

namespace lbgb {

constexpr int ADJ_VALUES = 5;  // dJ/d tau_A, tau_B, G, zeta_A, zeta_B

struct AdjArgs {
    const void* adj_in;   // lambda(t+1)
    void* adj_out;        // lambda(t)
    void* sbar;           // [2][3][N]: adjoint of S^k at fluid sites
    void* coef;           // [2][N]: per particle node, dJ/dpsi (1+zeta)/W
    void* coef_wall;      // [2 walls][2][nx ny]
    const double* dJdF;   // [nc][3] dJ/dF_liq of this step (device) or null
    double* red;          // block partials [blocks][ADJ_VALUES][2]
};

// E_i(rho, u) / rho = w_i (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)
template <typename C>
__device__ __forceinline__ C eq_shape(int i, C ux, C uy, C uz, C uu) {
    C cu = C(cx(i)) * ux + C(cy(i)) * uy + C(cz(i)) * uz;
    return wgt<C>(i) * (C(1) + C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu);
}

// weighted moments of an adjoint vector mu over the lattice:
// m0 = sum w mu, m1 = sum w mu c, m2 = sum w mu c c^T (xx, yy, zz, xy, xz, yz)
template <typename C>
struct Mom {
    C m0, m1[3], m2[6];
};

template <typename C>
__device__ __forceinline__ void moments_of(const C (&mu)[Q], Mom<C>& M) {
    M.m0 = 0;
    for (int d = 0; d < 3; d++) M.m1[d] = 0;
    for (int d = 0; d < 6; d++) M.m2[d] = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        C wm = wgt<C>(i) * mu[i];
        M.m0 += wm;
        M.m1[0] += C(cx(i)) * wm; M.m1[1] += C(cy(i)) * wm; M.m1[2] += C(cz(i)) * wm;
        M.m2[0] += C(cx(i) * cx(i)) * wm; M.m2[1] += C(cy(i) * cy(i)) * wm; M.m2[2] += C(cz(i) * cz(i)) * wm;
        M.m2[3] += C(cx(i) * cy(i)) * wm; M.m2[4] += C(cx(i) * cz(i)) * wm; M.m2[5] += C(cy(i) * cz(i)) * wm;
    }
}

// sum_i mu_i E_i(rho,u)/rho = m0 + 3 m1.u + 9/2 u^T m2 u - 3/2 u.u m0
template <typename C>
__device__ __forceinline__ C mom_shape(const Mom<C>& M, const C (&u)[3]) {
    C uMu = M.m2[0] * u[0] * u[0] + M.m2[1] * u[1] * u[1] + M.m2[2] * u[2] * u[2] +
            C(2) * (M.m2[3] * u[0] * u[1] + M.m2[4] * u[0] * u[2] + M.m2[5] * u[1] * u[2]);
    C uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return M.m0 + C(3) * (M.m1[0] * u[0] + M.m1[1] * u[1] + M.m1[2] * u[2]) + C(4.5) * uMu - C(1.5) * uu * M.m0;
}

// sum_i mu_i dE_i(rho,u)/du / rho = 3 m1 + 9 m2 u - 3 u m0
template <typename C>
__device__ __forceinline__ void mom_grad(const Mom<C>& M, const C (&u)[3], C (&g)[3]) {
    C m2u0 = M.m2[0] * u[0] + M.m2[3] * u[1] + M.m2[4] * u[2];
    C m2u1 = M.m2[3] * u[0] + M.m2[1] * u[1] + M.m2[5] * u[2];
    C m2u2 = M.m2[4] * u[0] + M.m2[5] * u[1] + M.m2[2] * u[2];
    g[0] = C(3) * M.m1[0] + C(9) * m2u0 - C(3) * u[0] * M.m0;
    g[1] = C(3) * M.m1[1] + C(9) * m2u1 - C(3) * u[1] * M.m0;
    g[2] = C(3) * M.m1[2] + C(9) * m2u2 - C(3) * u[2] * M.m0;
}

// sum over the block of one double per thread, written by thread 0 to *out
// (warp shuffles, then warps in order; blockDim.x a multiple of 32)
__device__ void block_sum_store(double v, double* out) {
    __shared__ double sh[32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
        *out = t;
    }
}

// Local adjoint of the collision and streaming at each fluid site.
template <int PREC>
__global__ void __launch_bounds__(128) k_adj_local(Lattice L, AdjArgs A) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y, z = blockIdx.z;
    C part[ADJ_VALUES] = {0, 0, 0, 0, 0};
    long long s = (long long)x + (long long)L.nx * ((long long)y + (long long)L.ny * z);
    const C* Lin = (const C*)A.adj_in;
    const C* Rin = Lin + 2 * Q * L.pstride;
    C* Lout = (C*)A.adj_out;
    C* sb = (C*)A.sbar;
    bool act = x < L.nx && !L.mask[s];
    if (act) {
        SiteNbr n = site_nbr(L, x, y, z);
        C fv[2][Q], rho[2], j[2][3], F[2][3], u[3], om;
        load_site<PREC>(L, (const S*)L.f_cur, s, fv, rho, j);
        // S^A, S^B (the force uses S of the other component)
        C SA[3] = {0, 0, 0}, SB[3] = {0, 0, 0};
        {
            const C* psi = (const C*)L.psi;
            const C* pw = (const C*)L.psi_wall;
            long long nxy = (long long)L.nx * L.ny;
#pragma unroll
            for (int i = 1; i < Q; i++) {
                C pa, pb;
                if (nbr_is_wall(n, i)) {
                    int X = cx(i) == 0 ? n.x : (cx(i) > 0 ? n.xp : n.xm);
                    int Y = cy(i) == 0 ? n.y : (cy(i) > 0 ? n.yp : n.ym);
                    int side = cz(i) < 0 ? 0 : 1;
                    long long w = (long long)X + (long long)L.nx * Y;
                    pa = pw[2 * (side * nxy + w)];
                    pb = pw[2 * (side * nxy + w) + 1];
                } else {
                    long long m = nbr_index(L, n, i);
                    pa = psi[2 * m];
                    pb = psi[2 * m + 1];
                }
                C w = wgt<C>(i);
                SA[0] += C(cx(i)) * w * pa; SA[1] += C(cy(i)) * w * pa; SA[2] += C(cz(i)) * w * pa;
                SB[0] += C(cx(i)) * w * pb; SB[1] += C(cy(i)) * w * pb; SB[2] += C(cz(i)) * w * pb;
            }
        }
        C G = C(L.P.G);
        for (int d = 0; d < 3; d++) {
            C g = C(L.P.body_force[d]);
            F[0][d] = -G * rho[0] * SB[d] + rho[0] * g;
            F[1][d] = -G * rho[1] * SA[d] + rho[1] * g;
        }
        mixture<C>(L, rho, j, u, om);
        C tiny = sizeof(C) == 8 ? C(1e-300) : C(1e-30);
        C v[2][3];
        for (int k = 0; k < 2; k++)
            for (int d = 0; d < 3; d++) v[k][d] = rho[k] > tiny ? u[d] + F[k][d] / rho[k] : u[d];
        C a = C(1) - om;
        // incoming adjoint mu = dJ/df*, and the wall bounce-back density term
        C mu[2][Q];
        C rbar[2] = {0, 0};
        const double* uwlo = L.P.wall_u_lo;
        const double* uwhi = L.P.wall_u_hi;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            if (i != 0 && nbr_is_wall(n, i)) {
                const double* uw = cz(i) < 0 ? uwlo : uwhi;
                C cu = C(cx(i) * uw[0] + cy(i) * uw[1] + cz(i) * uw[2]);
                for (int k = 0; k < 2; k++) {
                    C lam = Lin[((long long)(k * Q + opp(i))) * L.pstride + s] + Rin[k * L.pstride + s];
                    mu[k][i] = lam;
                    rbar[k] += lam * (-C(6) * wgt<C>(i) * cu);
                }
                continue;
            }
            long long m = i == 0 ? s : nbr_index(L, n, i);
            if (i == 0 || !L.mask[m]) {
                for (int k = 0; k < 2; k++)
                    mu[k][i] = Lin[((long long)(k * Q + i)) * L.pstride + m] + Rin[k * L.pstride + m];
            } else {
                // bounce-back on a fixed particle, plus the link force of Eq. 19
                C gc = 0;
                if (A.dJdF) {
                    const double* gp = A.dJdF + 3 * L.owner[m];
                    gc = C(2) * C(cx(i) * gp[0] + cy(i) * gp[1] + cz(i) * gp[2]);
                }
                for (int k = 0; k < 2; k++)
                    mu[k][i] = Lin[((long long)(k * Q + opp(i))) * L.pstride + s] + Rin[k * L.pstride + s] + gc;
            }
        }
        // backward through the collision
        C ubar[3] = {0, 0, 0}, abar = 0, Fbar[2][3];
        for (int k = 0; k < 2; k++) {
            Mom<C> M;
            moments_of<C>(mu[k], M);
            C P = 0;
#pragma unroll
            for (int i = 0; i < Q; i++) P += mu[k][i] * fv[k][i];
            C shu = mom_shape<C>(M, u), shv = mom_shape<C>(M, v[k]);
            abar += P - rho[k] * shu;
            rbar[k] += -a * shu + shv;
            C gu[3], gv[3];
            mom_grad<C>(M, u, gu);
            mom_grad<C>(M, v[k], gv);
            for (int d = 0; d < 3; d++) {
                ubar[d] += -a * rho[k] * gu[d];
                C vbar = rho[k] * gv[d];
                if (rho[k] > tiny) {
                    ubar[d] += vbar;
                    Fbar[k][d] = vbar / rho[k];
                    rbar[k] += -vbar * F[k][d] / (rho[k] * rho[k]);
                } else {
                    ubar[d] += vbar;
                    Fbar[k][d] = 0;
                }
            }
        }
        // forces: F^A = -G rho^A S^B + rho^A g, F^B = -G rho^B S^A + rho^B g
        C SAbar[3], SBbar[3], Gbar = 0;
        for (int d = 0; d < 3; d++) {
            C g = C(L.P.body_force[d]);
            rbar[0] += Fbar[0][d] * (-G * SB[d] + g);
            rbar[1] += Fbar[1][d] * (-G * SA[d] + g);
            SBbar[d] = -G * rho[0] * Fbar[0][d];
            SAbar[d] = -G * rho[1] * Fbar[1][d];
            Gbar += -rho[0] * Fbar[0][d] * SB[d] - rho[1] * Fbar[1][d] * SA[d];
        }
        // mixture velocity
        C w0 = C(1) / C(L.P.tau[0]), w1 = C(1) / C(L.P.tau[1]);
        C D = w0 * rho[0] + w1 * rho[1];
        C jbar[2][3];
        C udotub = ubar[0] * u[0] + ubar[1] * u[1] + ubar[2] * u[2];
        C Dbar = -udotub / D;
        for (int d = 0; d < 3; d++) {
            jbar[0][d] = w0 * ubar[d] / D;
            jbar[1][d] = w1 * ubar[d] / D;
        }
        rbar[0] += w0 * Dbar;
        rbar[1] += w1 * Dbar;
        C wbar0 = (ubar[0] * j[0][0] + ubar[1] * j[0][1] + ubar[2] * j[0][2]) / D + Dbar * rho[0];
        C wbar1 = (ubar[0] * j[1][0] + ubar[1] * j[1][1] + ubar[2] * j[1][2]) / D + Dbar * rho[1];
        C t0 = C(L.P.tau[0]), t1 = C(L.P.tau[1]);
        C taub0 = -wbar0 / (t0 * t0), taub1 = -wbar1 / (t1 * t1);
        // relaxation frequency of the mixture
        C nu0 = (t0 - C(0.5)) / C(3), nu1 = (t1 - C(0.5)) / C(3);
        C rt = rho[0] + rho[1];
        C q = (rho[0] / rt) / nu0 + (rho[1] / rt) / nu1;
        C nub = C(1) / q;
        C ombar = -abar;
        C nubbar = ombar * (-C(3) * om * om);
        C qbar = nubbar * (-nub * nub);
        rbar[0] += qbar * (C(1) / nu0 - q) / rt;
        rbar[1] += qbar * (C(1) / nu1 - q) / rt;
        taub0 += qbar * (-(rho[0] / rt) / (nu0 * nu0)) / C(3);
        taub1 += qbar * (-(rho[1] / rt) / (nu1 * nu1)) / C(3);
        // local adjoint of the populations
#pragma unroll
        for (int k = 0; k < 2; k++)
#pragma unroll
            for (int i = 0; i < Q; i++)
                Lout[((long long)(k * Q + i)) * L.pstride + s] =
                    a * mu[k][i] + rbar[k] + C(cx(i)) * jbar[k][0] + C(cy(i)) * jbar[k][1] + C(cz(i)) * jbar[k][2];
        for (int d = 0; d < 3; d++) {
            sb[(0 * 3 + d) * L.N + s] = SAbar[d];
            sb[(1 * 3 + d) * L.N + s] = SBbar[d];
        }
        part[0] = taub0;
        part[1] = taub1;
        part[2] = Gbar;
    }
    // block partials of the parameter gradients (FP64 across threads)
    int nb = gridDim.x * gridDim.y * gridDim.z;
    int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    for (int v = 0; v < 3; v++) block_sum_store(double(part[v]), A.red + (long long)v * nb + b);
}

// dJ/dpsi^k(y) = sum_i w_i c_i . Sbar^k(y - c_i) over fluid x = y - c_i.  On
// fluid nodes it is the density adjoint R; on particle frontier nodes it
// becomes coef = dJ/dpsi (1 + zeta^k) / W (W = sum of the fluid-neighbour
// weights, Eq. 20) and contributes dJ/dzeta^k = dJ/dpsi psi/(1 + zeta^k);
// with the Janus switch s of the node the factor is 1 + s_k zeta^k
// (s_A = s, s_B = -s) and the contribution dJ/dpsi s_k psi/(1 + s_k zeta^k).
template <int PREC>
__global__ void __launch_bounds__(128) k_adj_gather(Lattice L, AdjArgs A) {
    typedef typename Prec<PREC>::C C;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y, z = blockIdx.z;
    C zp[2] = {0, 0};
    if (x < L.nx) {
        long long s = (long long)x + (long long)L.nx * ((long long)y + (long long)L.ny * z);
        SiteNbr n = site_nbr(L, x, y, z);
        const C* sb = (const C*)A.sbar;
        C pb[2] = {0, 0}, W = 0;
#pragma unroll
        for (int i = 1; i < Q; i++) {
            // the site x = y - c_i is the neighbour along opp(i)
            int io = opp(i);
            if (nbr_is_wall(n, io)) continue;
            long long m = nbr_index(L, n, io);
            if (L.mask[m]) continue;
            C w = wgt<C>(i);
            W += w;
            for (int k = 0; k < 2; k++)
                pb[k] += w * (C(cx(i)) * sb[(k * 3 + 0) * L.N + m] + C(cy(i)) * sb[(k * 3 + 1) * L.N + m] +
                              C(cz(i)) * sb[(k * 3 + 2) * L.N + m]);
        }
        C* Rout = (C*)A.adj_out + 2 * Q * L.pstride;
        C* cf = (C*)A.coef;
        if (!L.mask[s]) {
            Rout[s] = pb[0];
            Rout[L.pstride + s] = pb[1];
        } else {
            const C* psi = (const C*)L.psi;
            // the node's wetting factors 1 + s_k zeta^k: s_k = 1 without the
            // Janus switch, s_A = s and s_B = -s with it
            C sk[2] = {C(1), C(1)};
            if (L.P.janus) {
                const int p = L.owner[s];
                const int xs[3] = {x, y, z}, Ls[3] = {L.nx, L.ny, L.nz};
                C d[3];
                for (int c = 0; c < 3; c++) {
                    double dd = (double)xs[c] - L.pos[3 * p + c];
                    if (L.per[c]) dd -= (double)Ls[c] * rint(dd / (double)Ls[c]);
                    d[c] = C(dd);
                }
                const C sw = janus_switch<C>(L, p, d);
                sk[0] = sw;
                sk[1] = -sw;
            }
            for (int k = 0; k < 2; k++) {
                C zk = C(1) + sk[k] * C(L.P.zeta[k]);
                cf[k * L.N + s] = W > C(0) ? pb[k] * zk / W : C(0);
                zp[k] = W > C(0) ? pb[k] * sk[k] * psi[2 * s + k] / zk : C(0);
            }
        }
    }
    int nb = gridDim.x * gridDim.y * gridDim.z;
    int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    for (int v = 0; v < 2; v++) block_sum_store(double(zp[v]), A.red + (long long)(3 + v) * nb + b);
}

// wall nodes: dJ/dpsi_wall from the fluid plane next to the wall, turned into
// coef_wall = dJ/dpsi_wall / W (the wall density is a plain mean)
template <typename C>
__global__ void k_adj_wall(Lattice L, AdjArgs A) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y, side = blockIdx.z;
    if (x >= L.nx) return;
    int zf = side == 0 ? 0 : L.nz - 1;
    int dz = side == 0 ? -1 : 1;  // links from the fluid plane into the wall
    const C* sb = (const C*)A.sbar;
    C pb[2] = {0, 0}, W = 0;
    long long nxy = (long long)L.nx * L.ny;
    for (int i = 1; i < Q; i++) {
        if (cz(i) != dz) continue;
        // fluid site x_f = wall site - c_i
        int X = x - cx(i), Y = y - cy(i);
        X = X < 0 ? X + L.nx : (X >= L.nx ? X - L.nx : X);
        Y = Y < 0 ? Y + L.ny : (Y >= L.ny ? Y - L.ny : Y);
        long long m = (long long)X + (long long)L.nx * ((long long)Y + (long long)L.ny * zf);
        if (L.mask[m]) continue;
        C w = wgt<C>(i);
        W += w;
        for (int k = 0; k < 2; k++)
            pb[k] += w * (C(cx(i)) * sb[(k * 3 + 0) * L.N + m] + C(cy(i)) * sb[(k * 3 + 1) * L.N + m] +
                          C(cz(i)) * sb[(k * 3 + 2) * L.N + m]);
    }
    C* cw = (C*)A.coef_wall;
    long long w = (long long)x + (long long)L.nx * y;
    for (int k = 0; k < 2; k++) cw[(side * 2 + k) * nxy + w] = W > C(0) ? pb[k] / W : C(0);
}

// fluid sites next to particle or wall nodes receive the virtual / wall
// density adjoint: R^k(x) += sum_j w_j coef^k(x + c_j)
template <int PREC>
__global__ void __launch_bounds__(128) k_adj_scatter(Lattice L, AdjArgs A) {
    typedef typename Prec<PREC>::C C;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y, z = blockIdx.z;
    if (x >= L.nx) return;
    long long s = (long long)x + (long long)L.nx * ((long long)y + (long long)L.ny * z);
    if (L.mask[s]) return;
    SiteNbr n = site_nbr(L, x, y, z);
    const C* cf = (const C*)A.coef;
    const C* cw = (const C*)A.coef_wall;
    long long nxy = (long long)L.nx * L.ny;
    C add[2] = {0, 0};
    bool any = false;
#pragma unroll
    for (int j = 1; j < Q; j++) {
        C w = wgt<C>(j);
        if (nbr_is_wall(n, j)) {
            int X = cx(j) == 0 ? n.x : (cx(j) > 0 ? n.xp : n.xm);
            int Y = cy(j) == 0 ? n.y : (cy(j) > 0 ? n.yp : n.ym);
            int side = cz(j) < 0 ? 0 : 1;
            long long wi = (long long)X + (long long)L.nx * Y;
            add[0] += w * cw[(side * 2 + 0) * nxy + wi];
            add[1] += w * cw[(side * 2 + 1) * nxy + wi];
            any = true;
            continue;
        }
        long long m = nbr_index(L, n, j);
        if (!L.mask[m]) continue;
        add[0] += w * cf[m];
        add[1] += w * cf[L.N + m];
        any = true;
    }
    if (!any) return;
    C* Rout = (C*)A.adj_out + 2 * Q * L.pstride;
    Rout[s] += add[0];
    Rout[L.pstride + s] += add[1];
}

// Sum of the block partials of each parameter gradient, added to the
// accumulator out[ADJ_VALUES]: warp v sums value v, lane l the partials
// l, l + 32, ... (Neumaier), then the lanes merge in a fixed order.
__global__ void k_adj_reduce(const double* red, int nb, double* out) {
    const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (v >= ADJ_VALUES) return;
    NSum t = {0.0, 0.0};
    for (int b = lane; b < nb; b += 32) t.add(red[(long long)v * nb + b]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        NSum o = {__shfl_down_sync(0xffffffffu, t.s, off), __shfl_down_sync(0xffffffffu, t.c, off)};
        if (lane < off) t.merge(o);
    }
    if (lane == 0) out[v] += t.value();
}

// dJ/dF_p for J = weight sum_p sqrt(|F_p|^2 + eps^2)
__global__ void k_drag_gradient(int n, const double* F, double weight, double eps, double* out) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double f0 = F[3 * p], f1 = F[3 * p + 1], f2 = F[3 * p + 2];
    double sc = weight / sqrt(f0 * f0 + f1 * f1 + f2 * f2 + eps * eps);
    out[3 * p] = sc * f0;
    out[3 * p + 1] = sc * f1;
    out[3 * p + 2] = sc * f2;
}

// Seed of the interface measure A = sum_x (1 - phi^2), phi = (rho_A - rho_B)/
// (rho_A + rho_B), over fluid nodes: L = 0, R^k = dA/drho^k, and block
// partials of A itself.
template <int PREC>
__global__ void __launch_bounds__(128) k_adj_seed_interface(Lattice L, void* adj, double* red, double weight) {
    typedef typename Prec<PREC>::C C;
    typedef typename Prec<PREC>::S S;
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double val = 0.0;
    if (s < L.N) {
        C* Lout = (C*)adj;
        C* Rout = Lout + 2 * Q * L.pstride;
        for (int q = 0; q < 2 * Q; q++) Lout[(long long)q * L.pstride + s] = 0;
        C r0 = 0, r1 = 0;
        if (!L.mask[s]) {
            C fv[2][Q], rho[2], j[2][3];
            load_site<PREC>(L, (const S*)L.f_cur, s, fv, rho, j);
            C rt = rho[0] + rho[1];
            C phi = (rho[0] - rho[1]) / rt;
            r0 = C(weight) * (-C(4) * phi * rho[1] / (rt * rt));
            r1 = C(weight) * (C(4) * phi * rho[0] / (rt * rt));
            val = double(C(1) - phi * phi);
        }
        Rout[s] = r0;
        Rout[L.pstride + s] = r1;
    }
    block_sum_store(val, red + blockIdx.x);
}

__global__ void k_sum_blocks(const double* red, int nb, double* out) {
    if (threadIdx.x != 0) return;
    NSum t = {0.0, 0.0};
    for (int b = 0; b < nb; b++) t.add(red[b]);
    out[0] = t.value();
}

// dJ/drho^k(0) = sum_i w_i lambda^k_i(0) for f(0) = f^eq(rho^k(0), 0) = w_i rho^k(0)
template <int PREC>
__global__ void k_adj_initial(Lattice L, const void* adj, double* grad) {
    typedef typename Prec<PREC>::C C;
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= L.N) return;
    const C* Lin = (const C*)adj;
    const C* Rin = Lin + 2 * Q * L.pstride;
    for (int k = 0; k < 2; k++) {
        double g = 0.0;
        if (!L.mask[s]) {
            C acc = 0;
            for (int i = 0; i < Q; i++) acc += wgt<C>(i) * Lin[((long long)(k * Q + i)) * L.pstride + s];
            g = double(acc + Rin[k * L.pstride + s]);
        }
        grad[k * L.N + s] = g;
    }
}

// ---------------------------------------------------------- launchers
#define DISPATCHA(prec, call)                                 \
    switch (prec) {                                           \
        case LB_FP64: { const int P = LB_FP64; call; break; } \
        case LB_FP32: { const int P = LB_FP32; call; break; } \
        default:      { const int P = LB_FP16; call; break; } \
    }

size_t adjoint_field_bytes(const Lattice& L, int prec) {
    size_t c = prec == LB_FP64 ? 8 : 4;
    return (size_t)(2 * Q + 2) * L.pstride * c;
}

size_t adjoint_scratch_bytes(const Lattice& L, int prec) {
    size_t c = prec == LB_FP64 ? 8 : 4;
    size_t nxy = (size_t)L.nx * L.ny;
    dim3 g((L.nx + 127) / 128, L.ny, L.nz);
    size_t nb = (size_t)g.x * g.y * g.z;
    size_t nb1 = (size_t)((L.N + 127) / 128);
    return 6 * L.N * c + 2 * L.N * c + 4 * nxy * c + (ADJ_VALUES * (nb > nb1 ? nb : nb1) + 16) * 8 + 4096;
}

static AdjArgs adj_args(const Lattice& L, int prec, const void* in, void* out, void* scratch,
                        const double* dJdF) {
    size_t c = prec == LB_FP64 ? 8 : 4;
    size_t nxy = (size_t)L.nx * L.ny;
    char* p = (char*)scratch;
    AdjArgs A;
    A.adj_in = in;
    A.adj_out = out;
    A.sbar = p; p += 6 * L.N * c;
    A.coef = p; p += 2 * L.N * c;
    A.coef_wall = p; p += 4 * nxy * c;
    p = (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    A.red = (double*)p;
    A.dJdF = dJdF;
    return A;
}

// one adjoint step; the 5 parameter gradients of this step are added to grads_dev
int launch_adjoint_step(const Lattice& L, int prec, const void* in, void* out, void* scratch,
                        const double* dJdF_dev, double* grads_dev, cudaStream_t st) {
    AdjArgs A = adj_args(L, prec, in, out, scratch, dJdF_dev);
    dim3 g((L.nx + 127) / 128, L.ny, L.nz);
    int bx = L.nx >= 128 ? 128 : ((L.nx + 31) / 32) * 32;
    dim3 gg((L.nx + bx - 1) / bx, L.ny, L.nz);
    int nb = gg.x * gg.y * gg.z;
    int n = 0;
    DISPATCHA(prec, (k_adj_local<P><<<gg, bx, 0, st>>>(L, A)));
    n++;
    if (!L.per[2]) {
        dim3 gw((L.nx + 127) / 128, L.ny, 2);
        if (prec == LB_FP64) k_adj_wall<double><<<gw, 128, 0, st>>>(L, A);
        else k_adj_wall<float><<<gw, 128, 0, st>>>(L, A);
        n++;
    } else {
        size_t c = prec == LB_FP64 ? 8 : 4;
        cudaMemsetAsync(A.coef_wall, 0, 4 * (size_t)L.nx * L.ny * c, st);
    }
    DISPATCHA(prec, (k_adj_gather<P><<<gg, bx, 0, st>>>(L, A)));
    DISPATCHA(prec, (k_adj_scatter<P><<<gg, bx, 0, st>>>(L, A)));
    k_adj_reduce<<<1, 32 * ADJ_VALUES, 0, st>>>(A.red, nb, grads_dev);
    (void)g;
    return n + 3;
}

int launch_adjoint_seed(const Lattice& L, int prec, void* adj, void* scratch, double weight, double* value_dev,
                        cudaStream_t st) {
    AdjArgs A = adj_args(L, prec, nullptr, adj, scratch, nullptr);
    int nb = (int)((L.N + 127) / 128);
    DISPATCHA(prec, (k_adj_seed_interface<P><<<nb, 128, 0, st>>>(L, adj, A.red, weight)));
    k_sum_blocks<<<1, 32, 0, st>>>(A.red, nb, value_dev);
    return 2;
}

int launch_drag_gradient(int n, const double* F, double weight, double eps, double* out, cudaStream_t st) {
    if (n <= 0) return 0;
    k_drag_gradient<<<(n + 127) / 128, 128, 0, st>>>(n, F, weight, eps, out);
    return 1;
}

int launch_adjoint_initial(const Lattice& L, int prec, const void* adj, double* grad, cudaStream_t st) {
    DISPATCHA(prec, (k_adj_initial<P><<<(unsigned)((L.N + 255) / 256), 256, 0, st>>>(L, adj, grad)));
    return 1;
}

}  // namespace lbgb
