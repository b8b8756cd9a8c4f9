// One-component fluid: the LBGK fluid of a single species on D3Q19 without
// particles, the lattice of the paper's single-component benchmark (Sec. 5.1,
// first benchmark table; App. D benchmark test 1: one component, tau = 1,
// periodic).  The step is Eqs. 5-7 and 16 for one component, with the body
// force of the exact-difference source (Eq. 15, F = rho g) and no Shan-Chen
// force, and push streaming (Eq. 3) with the halfway bounce-back of moving
// walls (Eq. 9) on the z faces.
//
// Populations: element SKEW + s - c_ix of plane i (pop1_index), the skewed
// layout of the two-component lattice with one component, so that the 32
// pushes of a warp along one link fill whole aligned lines.  One thread per
// site, 19 loads and 19 stores: the kernel needs no staging.
#include "lbgb_internal.cuh"

namespace lbgb {

__host__ __device__ constexpr long long pop1_index(int i, long long s, long long pstride) {
    return (long long)i * pstride + SKEW + s - cx(i);
}

// f = f^eq(rho, u) from the FP64 stage (rho^A [N], rho^B [N] (unused), u [3][N])
template <int PREC>
__global__ void k1_init(Lattice L, const double* __restrict__ stage) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= L.N) return;
    const C r = C(stage[s]);
    const C ux = C(stage[2 * L.N + s]), uy = C(stage[3 * L.N + s]), uz = C(stage[4 * L.N + s]);
    const C uu = ux * ux + uy * uy + uz * uz;
    S* f = (S*)L.f_cur;
#pragma unroll
    for (int i = 0; i < Q; i++) st_pop(f + pop1_index(i, s, L.pstride), feq<C>(i, r, ux, uy, uz, uu), pop_shift<S, C>(L, 0, i));
}

// rho of node s from f(t)
template <int PREC>
__device__ __forceinline__ typename Prec<PREC>::C node_rho1(const Lattice& L, long long s) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    const S* f = (const S*)L.f_cur;
    C r = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) r += ld_pop(f + pop1_index(i, s, L.pstride), pop_shift<S, C>(L, 0, i));
    return r;
}

// rho_w of the velocity faces (Eq. 9) extrapolated to first order from the
// boundary node b and the next interior node b + 1 along z (Sec. 2.2),
// rho_w = rho_b + (rho_b - rho_{b+1}) / 2 (rho_b alone for nz < 2), one
// thread per column of face blockIdx.z, into element 0 of the face record
template <int PREC>
__global__ void k1_face_values(Lattice L) {
    typedef typename Prec<PREC>::C C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, side = blockIdx.z;
    if (x >= L.nx || L.P.open[side] != 2) return;
    const long long nxy = (long long)L.nx * L.ny, col = (long long)x + (long long)L.nx * y;
    const int zb = side == 0 ? 0 : L.nz - 1, zi = side == 0 ? 1 : L.nz - 2;
    C r = node_rho1<PREC>(L, col + nxy * zb);
    if (zi >= 0 && zi < L.nz) r += C(0.5) * (r - node_rho1<PREC>(L, col + nxy * zi));
    ((C*)L.face)[5 * (side * nxy + col)] = r;
}

// One time step of every site (grid: x chunks, y, z).  UNIT: omega = 1, so
// Eq. 16 is f* = f^eq(rho, u + g) and the populations enter only through
// their moments.
template <int PREC, bool UNIT, bool SR>
__global__ void __launch_bounds__(128) k1_step(Lattice L) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= L.nx) return;
    const int nx = L.nx, nxy = L.nx * L.ny;
    const unsigned s = (unsigned)x + (unsigned)nx * ((unsigned)y + (unsigned)L.ny * (unsigned)z);
    const long long ps = L.pstride;
    const S* fc = (const S*)L.f_cur;
    C f[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) f[i] = ld_pop(fc + pop1_index(i, s, ps), pop_shift<S, C>(L, 0, i));
    // Eqs. 6, 7
    C rho = 0, j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < Q; i++) {
        rho += f[i];
        if (cx(i)) j[0] += C(cx(i)) * f[i];
        if (cy(i)) j[1] += C(cy(i)) * f[i];
        if (cz(i)) j[2] += C(cz(i)) * f[i];
    }
    if (!(rho > C(0) && rho < C(1e30))) atomicOr(L.flags, FLAG_NONFINITE);
    const C ir = C(1) / rho;
    C u[3], us[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        u[d] = j[d] * ir;
        us[d] = u[d] + prm<C>(L.P.body_force[d], L.PF.body_force[d]);  // u + F / rho, F = rho g
    }
    const C uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const C uus = us[0] * us[0] + us[1] * us[1] + us[2] * us[2];
    const C om = prm<C>(L.inv_tau[0], L.PF.inv_tau[0]);
    // Eq. 16: f* = f + omega (f^eq(rho, u) - f) + f^eq(rho, u + F/rho) - f^eq(rho, u)
    C fs[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        if (UNIT)
            fs[i] = feq<C>(i, rho, us[0], us[1], us[2], uus);
        else
            fs[i] = (C(1) - om) * (f[i] - feq<C>(i, rho, u[0], u[1], u[2], uu)) + feq<C>(i, rho, us[0], us[1], us[2], uus);
    }
    // push (Eq. 3) to the pair element SKEW + q - c_ix of the destination q,
    // whose c_ix shift the skew cancels; across a z wall the own element of
    // plane opp(i), f_ibar = f*_i - 6 w_i rho c_i.u_w (Eq. 9)
    const int wxp = x == nx - 1 ? -nx : 0, wxm = x == 0 ? nx : 0;
    const int dyp = y == L.ny - 1 ? nx - nxy : nx, dym = y == 0 ? nxy - nx : -nx;
    const int dzp = z == L.nz - 1 ? nxy - (int)L.N : nxy, dzm = z == 0 ? (int)L.N - nxy : -nxy;
    const bool wall_lo = z == 0 && !L.per[2], wall_hi = z == L.nz - 1 && !L.per[2];
    S* fn = (S*)L.f_nxt;
    C val[Q];
    long long dst[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const bool wall = (cz(i) < 0 && wall_lo) || (cz(i) > 0 && wall_hi);
        const int off = (cx(i) > 0 ? wxp : (cx(i) < 0 ? wxm : 0)) + (cy(i) > 0 ? dyp : (cy(i) < 0 ? dym : 0)) +
                        (cz(i) > 0 ? dzp : (cz(i) < 0 ? dzm : 0));
        C v = fs[i];
        long long e = (long long)i * ps + SKEW + (long long)s + off;
        if (wall) {
            const double* uwd = cz(i) < 0 ? L.P.wall_u_lo : L.P.wall_u_hi;
            const float* uwf = cz(i) < 0 ? L.PF.wall_u_lo : L.PF.wall_u_hi;
            const C cw = C(cx(i)) * prm<C>(uwd[0], uwf[0]) + C(cy(i)) * prm<C>(uwd[1], uwf[1]) +
                         C(cz(i)) * prm<C>(uwd[2], uwf[2]);
            // rho_w: rho of this node, or on a velocity face with
            // extrapolation the face value of the column (k1_face_values)
            const int h = cz(i) < 0 ? 0 : 1;
            C rw = rho;
            if (L.P.open_extrap && L.P.open[h] == 2)
                rw = ((const C*)L.face)[5 * ((long long)h * nxy + x + (long long)nx * y)];
            v = fs[i] - C(6) * wgt<C>(i) * rw * cw;
            e = (long long)opp(i) * ps + SKEW + (long long)s + cx(i);
        }
        val[i] = v;
        dst[i] = e;
    }
    if constexpr (SR) {
        // two populations per stochastic-rounding conversion (the helper
        // packs B in the upper half: here link i + 1)
        unsigned rs = sr_start(s, L.sr_key);
#pragma unroll
        for (int i = 0; i < Q; i += 2) {
            const int i2 = i + 1 < Q ? i + 1 : i;
            const unsigned d = cvt_sr_pair(val[i], val[i2], pop_shift<S, C>(L, 0, i), pop_shift<S, C>(L, 0, i2),
                                           sr_next2(rs));
            *reinterpret_cast<unsigned short*>(fn + dst[i]) = (unsigned short)(d & 0xffffu);
            if (i + 1 < Q) *reinterpret_cast<unsigned short*>(fn + dst[i2]) = (unsigned short)(d >> 16);
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; i++) st_pop(fn + dst[i], val[i], pop_shift<S, C>(L, 0, i));
    }
}

// rho, 0 and u = (j + F/2) / rho (end of Sec. 2.3) into the FP64 stage [5][N]
template <int PREC>
__global__ void k1_fields_out(Lattice L, double* __restrict__ stage) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= L.N) return;
    const S* f = (const S*)L.f_cur;
    C rho = 0, j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const C v = ld_pop(f + pop1_index(i, s, L.pstride), pop_shift<S, C>(L, 0, i));
        rho += v;
        if (cx(i)) j[0] += C(cx(i)) * v;
        if (cy(i)) j[1] += C(cy(i)) * v;
        if (cz(i)) j[2] += C(cz(i)) * v;
    }
    stage[s] = double(rho);
    stage[L.N + s] = 0.0;
    for (int d = 0; d < 3; d++)
        stage[(2 + d) * L.N + s] = double((j[d] + C(0.5) * rho * prm<C>(L.P.body_force[d], L.PF.body_force[d])) / rho);
}

// block partial sums of mass, j and j + F/2 in the layout of the
// two-component totals (the mass of component B is zero)
template <int PREC>
__global__ void __launch_bounds__(256) k1_totals_partial(Lattice L) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    NSum acc[8];
    for (int a = 0; a < 8; a++) acc[a].s = acc[a].c = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < L.N; s += stride) {
        const S* f = (const S*)L.f_cur;
        C rho = 0, j[3] = {0, 0, 0};
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const C v = ld_pop(f + pop1_index(i, s, L.pstride), pop_shift<S, C>(L, 0, i));
            rho += v;
            if (cx(i)) j[0] += C(cx(i)) * v;
            if (cy(i)) j[1] += C(cy(i)) * v;
            if (cz(i)) j[2] += C(cz(i)) * v;
        }
        acc[0].add(double(rho));
        for (int d = 0; d < 3; d++) {
            acc[2 + d].add(double(j[d]));
            acc[5 + d].add(double(j[d] + C(0.5) * rho * prm<C>(L.P.body_force[d], L.PF.body_force[d])));
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

template <int PREC>
__global__ void k1_pops_out(Lattice L, int i, double* __restrict__ stage) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= L.N) return;
    stage[s] = double(ld_pop((const S*)L.f_cur + pop1_index(i, s, L.pstride), pop_shift<S, C>(L, 0, i)));
}

// ------------------------------------------------------------ launchers
#define DISPATCH1(prec, call)                                 \
    switch (prec) {                                           \
        case LB_FP64: { const int P = LB_FP64; call; break; } \
        case LB_FP32: { const int P = LB_FP32; call; break; } \
        default:      { const int P = LB_FP16; call; break; } \
    }

static inline unsigned nblk1(long long n, int b) { return (unsigned)((n + b - 1) / b); }

int launch_single_init(const Lattice& L, int prec, const double* stage, cudaStream_t st) {
    DISPATCH1(prec, (k1_init<P><<<nblk1(L.N, 256), 256, 0, st>>>(L, stage)));
    return 1;
}

int launch_single_face_values(const Lattice& L, int prec, cudaStream_t st) {
    if (L.per[2] || !L.P.open_extrap || (L.P.open[0] != 2 && L.P.open[1] != 2)) return 0;
    dim3 g((unsigned)((L.nx + 127) / 128), (unsigned)L.ny, 2);
    DISPATCH1(prec, (k1_face_values<P><<<g, 128, 0, st>>>(L)));
    return 1;
}

int launch_single_step(const Lattice& L, int prec, cudaStream_t st) {
    const int bx = L.nx >= 128 ? 128 : ((L.nx + 31) / 32) * 32;
    const dim3 g((unsigned)((L.nx + bx - 1) / bx), (unsigned)L.ny, (unsigned)L.nz);
    const bool unit = L.P.tau[0] == 1.0;
    if (prec == LB_FP16 && L.sr) {
        if (unit) k1_step<LB_FP16, true, true><<<g, bx, 0, st>>>(L);
        else k1_step<LB_FP16, false, true><<<g, bx, 0, st>>>(L);
        return 1;
    }
    if (unit) {
        DISPATCH1(prec, (k1_step<P, true, false><<<g, bx, 0, st>>>(L)));
    } else {
        DISPATCH1(prec, (k1_step<P, false, false><<<g, bx, 0, st>>>(L)));
    }
    return 1;
}

int launch_single_fields_out(const Lattice& L, int prec, double* stage, cudaStream_t st) {
    DISPATCH1(prec, (k1_fields_out<P><<<nblk1(L.N, 256), 256, 0, st>>>(L, stage)));
    return 1;
}

int launch_single_totals_partial(const Lattice& L, int prec, cudaStream_t st) {
    DISPATCH1(prec, (k1_totals_partial<P><<<L.red_blocks, 256, 0, st>>>(L)));
    return 1;
}

int launch_single_populations_out(const Lattice& L, int prec, int i, double* stage, cudaStream_t st) {
    DISPATCH1(prec, (k1_pops_out<P><<<nblk1(L.N, 256), 256, 0, st>>>(L, i, stage)));
    return 1;
}

}  // namespace lbgb
