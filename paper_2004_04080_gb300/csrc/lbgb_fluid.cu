// lbgb_fluid.cu -- lattice kernels: initialisation, densities, the fused
// collide + Shan-Chen + bounce-back + push-stream step, and read-outs.
//
// Populations are stored structure-of-arrays, f[k][i][s] (component k, link
// i, site s = x + nx (y + ny z)), with the population planes padded to a
// multiple of 64 sites.  The state between time steps is the post-streaming
// population f(t) (the paper's step starts from it, Sec. 3.1); one step
// reads f(t) at each site, collides locally and pushes f*(t) to the
// neighbours, writing f(t+1) into the second buffer.
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
            st_pop(f + ((long long)(k * Q + i)) * L.pstride + s, feq<C>(i, r, ux, uy, uz, uu),
                   pop_shift<S, C>(L, k, i));
    }
}

// rho^k on fluid nodes (0 on particle nodes) into psi; flags non-finite or
// negative densities.
template <int PREC>
__global__ void k_density(Lattice L) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= L.N) return;
    C* psi = (C*)L.psi;
    if (L.mask[s]) {
        psi[s] = 0;
        psi[L.N + s] = 0;
        return;
    }
    const S* f = (const S*)L.f_cur;
    C rho[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        C r = 0;
#pragma unroll
        for (int i = 0; i < Q; i++)
            r += ld_pop(f + ((long long)(k * Q + i)) * L.pstride + s, pop_shift<S, C>(L, k, i));
        rho[k] = r;
        psi[k * L.N + s] = r;
    }
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
        num0 += w * psi[m];
        num1 += w * psi[L.N + m];
        den += w;
    }
    long long w = (long long)x + (long long)L.nx * y;
    pw[(side * 2 + 0) * nxy + w] = den > C(0) ? num0 / den : C(0);
    pw[(side * 2 + 1) * nxy + w] = den > C(0) ? num1 / den : C(0);
}

// The fused step at one fluid site: moments (Eqs. 6, 7, 14), Shan-Chen force
// (Eq. 11), EDM collision (Eq. 16), then push-streaming (Eq. 3) with halfway
// bounce-back on particle links (Eq. 17, wall velocity of Eq. 18) and on wall
// links (Eq. 9).  Particle velocities are the stored v(t-1/2), omega(t-1/2).
template <int PREC>
__global__ void __launch_bounds__(128) k_collide_push(Lattice L) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y, z = blockIdx.z;
    if (x >= L.nx) return;
    long long s = (long long)x + (long long)L.nx * ((long long)y + (long long)L.ny * z);
    if (L.mask[s]) return;
    SiteNbr n = site_nbr(L, x, y, z);
    C fv[2][Q], rho[2], j[2][3], F[2][3], u[3], om;
    load_site<PREC>(L, (const S*)L.f_cur, s, fv, rho, j);
    sc_force<C>(L, n, rho, F);
    mixture<C>(L, rho, j, u, om);
    C us[2][3];
    C tiny = sizeof(C) == 8 ? C(1e-300) : C(1e-30);
#pragma unroll
    for (int k = 0; k < 2; k++)
#pragma unroll
        for (int d = 0; d < 3; d++) us[k][d] = rho[k] > tiny ? u[d] + F[k][d] / rho[k] : u[d];
    C uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    C uus[2] = {us[0][0] * us[0][0] + us[0][1] * us[0][1] + us[0][2] * us[0][2],
                us[1][0] * us[1][0] + us[1][1] * us[1][1] + us[1][2] * us[1][2]};
    C one_m_om = C(1) - om;
    S* fn = (S*)L.f_nxt;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        C fs[2];
#pragma unroll
        for (int k = 0; k < 2; k++)
            fs[k] = one_m_om * (fv[k][i] - feq<C>(i, rho[k], u[0], u[1], u[2], uu)) +
                    feq<C>(i, rho[k], us[k][0], us[k][1], us[k][2], uus[k]);
        if (i != 0 && nbr_is_wall(n, i)) {
            const double* uw = cz(i) < 0 ? L.P.wall_u_lo : L.P.wall_u_hi;
            C cu = C(cx(i) * uw[0] + cy(i) * uw[1] + cz(i) * uw[2]);
#pragma unroll
            for (int k = 0; k < 2; k++)
                st_pop(fn + ((long long)(k * Q + opp(i))) * L.pstride + s,
                       fs[k] - C(6) * wgt<C>(i) * rho[k] * cu, pop_shift<S, C>(L, k, opp(i)));
            continue;
        }
        long long m = i == 0 ? s : nbr_index(L, n, i);
        if (i == 0 || !L.mask[m]) {
#pragma unroll
            for (int k = 0; k < 2; k++)
                st_pop(fn + ((long long)(k * Q + i)) * L.pstride + m, fs[k], pop_shift<S, C>(L, k, i));
        } else {
            // particle link: u_w = v_p + omega_p x (r_w - r_p), r_w = x + c_i/2
            int p = L.owner[m];
            double r[3] = {x + 0.5 * cx(i) - L.pos[3 * p], y + 0.5 * cy(i) - L.pos[3 * p + 1],
                           z + 0.5 * cz(i) - L.pos[3 * p + 2]};
            int Ls[3] = {L.nx, L.ny, L.nz};
#pragma unroll
            for (int d = 0; d < 3; d++)
                if (L.per[d]) r[d] -= Ls[d] * floor(r[d] / Ls[d] + 0.5);
            const double* v = L.vel + 3 * p;
            const double* w = L.omg + 3 * p;
            double uw0 = v[0] + (w[1] * r[2] - w[2] * r[1]);
            double uw1 = v[1] + (w[2] * r[0] - w[0] * r[2]);
            double uw2 = v[2] + (w[0] * r[1] - w[1] * r[0]);
            C cu = C(cx(i) * uw0 + cy(i) * uw1 + cz(i) * uw2);
#pragma unroll
            for (int k = 0; k < 2; k++)
                st_pop(fn + ((long long)(k * Q + opp(i))) * L.pstride + s,
                       fs[k] - C(6) * wgt<C>(i) * rho[k] * cu, pop_shift<S, C>(L, k, opp(i)));
        }
    }
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
    stage[s] = double(ld_pop(f + ((long long)(k * Q + i)) * L.pstride + s, pop_shift<S, C>(L, k, i)));
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
    DISPATCH(prec, (k_density<P><<<nblk(L.N, 256), 256, 0, st>>>(L)));
    return 1;
}

int launch_wall_psi(const Lattice& L, int prec, cudaStream_t st) {
    if (L.per[2]) return 0;
    dim3 g((unsigned)((L.nx + 127) / 128), (unsigned)L.ny, 2);
    if (prec == LB_FP64) k_wall_psi<double><<<g, 128, 0, st>>>(L);
    else k_wall_psi<float><<<g, 128, 0, st>>>(L);
    return 1;
}

int launch_fluid_step(const Lattice& L, int prec, cudaStream_t st) {
    int bx = site_bx(L);
    DISPATCH(prec, (k_collide_push<P><<<site_grid(L, bx), bx, 0, st>>>(L)));
    return 1;
}

int launch_fields_out(const Lattice& L, int prec, double* stage, cudaStream_t st) {
    int bx = site_bx(L);
    DISPATCH(prec, (k_fields_out<P><<<site_grid(L, bx), bx, 0, st>>>(L, stage)));
    return 1;
}

int launch_totals(const Lattice& L, int prec, double* out_dev, cudaStream_t st) {
    DISPATCH(prec, (k_totals_partial<P><<<L.red_blocks, 256, 0, st>>>(L)));
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
