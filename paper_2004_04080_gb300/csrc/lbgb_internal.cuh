// lbgb_internal.cuh -- device-side definitions shared by the library's
// translation units: the D3Q19 lattice as compile-time functions, storage
// conversions, the context layout and the kernel entry points.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/lbgb.h"

namespace lbgb {

// ---------------------------------------------------------------- lattice
// D3Q19 (Sec. 2.1).  Link 0 rests; 1-6 are the axis links +x,-x,+y,-y,+z,-z;
// 7-18 the face diagonals, ordered so that link i (odd) and i+1 are opposite.
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// The link vector of a link index known only at run time, from packed
// 2-bit fields (c + 1 of links 0..18), without a table in memory.
constexpr unsigned long long pack_c(int a) {
    unsigned long long v = 0;
    for (int i = 0; i < 19; i++)
        v |= (unsigned long long)((a == 0 ? cx(i) : (a == 1 ? cy(i) : cz(i))) + 1) << (2 * i);
    return v;
}
__device__ __forceinline__ int rc(int a, int i) {
    const unsigned long long P = a == 0 ? pack_c(0) : (a == 1 ? pack_c(1) : pack_c(2));
    return (int)((P >> (2 * i)) & 3ull) - 1;
}

// Link classes of a site (the word nb[s] the lean kernel reads, rebuilt
// around every node the remap changes): bit 0 the site is a particle node;
// bit i (1..18) the neighbour along c_i has the other kind (particle node
// next to fluid), never across a wall; NB_MULTI on a fluid site whose
// particle neighbours belong to more than one particle.
constexpr uint32_t NB_SOLID = 1u, NB_LINKS = 0x7FFFEu, NB_MULTI = 1u << 19;
constexpr int NB_CHG_CAP = 1 << 20;  // changed nodes listed per step (more: a full rebuild)

// lattice weights w0 = 1/3, w1-6 = 1/18, w7-18 = 1/36
template <typename C>
__host__ __device__ constexpr C wgt(int i) {
    return i == 0 ? C(1) / C(3) : (i <= 6 ? C(1) / C(18) : C(1) / C(36));
}
constexpr int Q = 19;

// Population storage.  Plane i holds the populations of link i of both
// components, side by side: the pair (f^A_i, f^B_i) of site s is pair
// SKEW + s - c_ix of plane i (elements 2 (i pstride + SKEW + s - c_ix) + k),
// s = x + nx (y + ny z).  A push along c_i (Eq. 3) from site s then writes
// the destination's pair at the source's x, so the 32 pushes of a warp's row
// fill whole aligned lines of the destination row, one vector store per
// link for both components.  Writes shifted by one pair instead left partial
// 32-byte sectors at both ends of every row segment, which halved the store
// bandwidth (DRAM read-modify-writes); the reads of a site's own
// populations, shifted by one pair now, cost nothing measurable.  Each plane
// is padded by SKEW = 64 pairs at both ends, which keeps the first site of
// every plane on a 256-byte boundary in each storage type.
constexpr long long SKEW = 64;
__host__ __device__ constexpr long long pop_index(int q, long long s, long long pstride) {
    return 2 * ((long long)(q % Q) * pstride + SKEW + s - cx(q % Q)) + q / Q;
}
// the element of component A of link i of site s (component B follows it)
__host__ __device__ constexpr long long pair_index(int i, long long s, long long pstride) {
    return 2 * ((long long)i * pstride + SKEW + s - cx(i));
}

// ---------------------------------------------------------- precisions
// Storage type S and compute type C of the populations.
template <int PREC> struct Prec;
template <> struct Prec<LB_FP64> { typedef double S; typedef double C; };
template <> struct Prec<LB_FP32> { typedef float S; typedef float C; };
template <> struct Prec<LB_FP16> { typedef __half S; typedef float C; };

// load / store one population; FP16 stores the deviation f - w_i rho0^k
__device__ __forceinline__ double ld_pop(const double* p, double) { return *p; }
__device__ __forceinline__ float ld_pop(const float* p, float) { return *p; }
__device__ __forceinline__ float ld_pop(const __half* p, float shift) {
    return __half2float(*p) + shift;
}
__device__ __forceinline__ void st_pop(double* p, double v, double) { *p = v; }
__device__ __forceinline__ void st_pop(float* p, float v, float) { *p = v; }
__device__ __forceinline__ void st_pop(__half* p, float v, float shift) {
    *p = __float2half_rn(v - shift);
}

// load / store the pair of one link of a site (p: component A, 8-, 4- or
// 16-byte aligned for FP32, FP16, FP64)
__device__ __forceinline__ void ld_pair(const double* p, double, double, double& a, double& b) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void ld_pair(const float* p, float, float, float& a, float& b) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void ld_pair(const __half* p, float sa, float sb, float& a, float& b) {
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
    a = v.x + sa;
    b = v.y + sb;
}
__device__ __forceinline__ void st_pair(double* p, double a, double b, double, double) {
    *reinterpret_cast<double2*>(p) = make_double2(a, b);
}
__device__ __forceinline__ void st_pair(float* p, float a, float b, float, float) {
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
__device__ __forceinline__ void st_pair(__half* p, float a, float b, float sa, float sb) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a - sa, b - sb);
}

// The same stores under a per-lane predicate, as predicated store
// instructions (a branch around a store diverges the warp and costs
// reconvergence instructions in every unrolled link).
__device__ __forceinline__ void st_pop_if(double* p, double v, double, bool on) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.f64 [%0], %1;\n\t}" ::"l"(p), "d"(v),
                 "r"((unsigned)on));
}
__device__ __forceinline__ void st_pop_if(float* p, float v, float, bool on) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.f32 [%0], %1;\n\t}" ::"l"(p), "f"(v),
                 "r"((unsigned)on));
}
__device__ __forceinline__ void st_pop_if(__half* p, float v, float shift, bool on) {
    const unsigned short h = __half_as_ushort(__float2half_rn(v - shift));
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.b16 [%0], %1;\n\t}" ::"l"(p), "h"(h),
                 "r"((unsigned)on));
}
__device__ __forceinline__ void st_pair_if(double* p, double a, double b, double, double, bool on) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q st.global.v2.f64 [%0], {%1, %2};\n\t}" ::"l"(p),
                 "d"(a), "d"(b), "r"((unsigned)on));
}
__device__ __forceinline__ void st_pair_if(float* p, float a, float b, float, float, bool on) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q st.global.v2.f32 [%0], {%1, %2};\n\t}" ::"l"(p),
                 "f"(a), "f"(b), "r"((unsigned)on));
}
__device__ __forceinline__ void st_pair_if(__half* p, float a, float b, float sa, float sb, bool on) {
    const __half2 v = __floats2half2_rn(a - sa, b - sb);  // A in the low half
    const unsigned h = *reinterpret_cast<const unsigned*>(&v);
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.b32 [%0], %1;\n\t}" ::"l"(p), "r"(h),
                 "r"((unsigned)on));
}

// Stochastic rounding of the FP16 deviation stores.  The two components of
// a link are converted together by the hardware's stochastic-rounding
// conversion to a pair of halves (cvt.rs.f16x2.f32: component B in the upper
// half, rounded with random bits 31..16, component A in the lower half with
// bits 15..0, which is the order of the pair in memory; each value rounds
// up with probability equal to its position between the two neighbouring
// half values, so the expected stored value is the FP32 one; subnormal
// halves included).  The random bits of a site start
// from Appleby's MurmurHash3 32-bit finaliser of (site, step key) and advance
// by the linear congruential step of Numerical Recipes (a = 1664525,
// c = 1013904223); each component takes the upper 16 bits of its own step
// (the low bits of such a generator are weak, and bits for several stores
// sliced from one product are correlated across a site's populations).
__device__ __forceinline__ unsigned sr_start(unsigned site, unsigned key) {
    unsigned h = site * 0x9E3779B1u ^ key;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}
// 32 random bits for one pair of stores: the upper halves of two steps
__device__ __forceinline__ unsigned sr_next2(unsigned& st) {
    st = st * 1664525u + 1013904223u;
    const unsigned hi = st & 0xffff0000u;
    st = st * 1664525u + 1013904223u;
    return hi | (st >> 16);
}
__device__ __forceinline__ unsigned cvt_sr_pair(float va, float vb, float sa, float sb, unsigned bits) {
    unsigned d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(vb - sb), "f"(va - sa), "r"(bits));
    return d;
}
__device__ __forceinline__ void st_pair_sr(__half* p, float va, float vb, float sa, float sb, unsigned bits) {
    *reinterpret_cast<unsigned*>(p) = cvt_sr_pair(va, vb, sa, sb, bits);
}
__device__ __forceinline__ void st_pair_sr_if(__half* p, float va, float vb, float sa, float sb, unsigned bits,
                                              bool on) {
    const unsigned d = cvt_sr_pair(va, vb, sa, sb, bits);
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.b32 [%0], %1;\n\t}" ::"l"(p), "r"(d),
                 "r"((unsigned)on));
}

// ------------------------------------------------------------- context
// FP32 copies of the lattice parameters the per-site arithmetic reads: the
// FP32 forms take these (a conversion from FP64 runs on the FP64 pipe, a
// small fraction of the FP32 rate), the FP64 form the FP64 originals.
struct ParamsF {
    float G, body_force[3], rho0[2], wall_u_lo[3], wall_u_hi[3], inv_tau[2], inv_nu[2];
};

template <typename C>
__device__ __forceinline__ C prm(double d, float f);
template <>
__device__ __forceinline__ double prm<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float prm<float>(double, float f) { return f; }

// Device-visible view of one lattice (passed by value to every kernel).
struct Lattice {
    int nx, ny, nz;
    int ncomp;         // 2: the two-component lattice; 1: one fluid component, no particles (lbgb_single.cu)
    long long N;       // nx*ny*nz
    long long pstride; // component pairs in a population plane (>= N, padded)
    int per[3];        // periodic flags
    void* f_cur;       // populations at time t: [19][pstride][2] of S (pair_index)
    void* f_nxt;       // populations at time t+1
    void* psi;         // [N][2] of C: (psi^A, psi^B) of a site side by side; rho^k on fluid, virtual density on frontier
    void* psi_wall;    // [2 walls][nx*ny][2 comps] of C (pairs, like psi)
    void* face;        // [2 faces][nx*ny][5] of C: rho_w^A, rho_w^B, u_w of the open faces
                       // extrapolated to first order (k_face_values; with P.open_extrap)
    uint8_t* mask;     // 1 on particle nodes
    int* owner;        // -1 fluid, else particle index
    int* evt;          // remap events: 4 (p+1) + 1 destroy, 4 (p+1) + 2 create
    uint32_t* nb;      // link classes of every site (NB_*), kept with the node map
    int* nb_chg;       // [0] count of the nodes the remap changed, list from [8] (NB_CHG_CAP)
    int* flags;        // [0] error bits
    // particles (FP64, [n][3] / [n][4] / [n])
    int nc;
    double *pos, *vel, *omg, *quat, *rad, *mass;
    double *Fliq, *Tliq, *Fliq_prev, *Tliq_prev;
    int* prev_valid;
    double *Fd, *Td, *Fc, *Tc, *Fs, *Ts, *Fpair, *Ftot, *Ttot;
    // fixed-point sums of the per-site terms of one step (see acc_add):
    // [ACC_TERMS][maxc][3][2] words, zeroed at the start of each step
    unsigned long long* acc;
    // particle pair list: [maxc][PAIR_LIST_MAX] neighbours sorted by index,
    // their count, the positions at the last build, the rebuild flag and the
    // count of builds
    int* vl_nb;
    int* vl_cnt;
    double* vl_ref;
    int* vl_flag;
    unsigned long long* vl_builds;
    int maxc;
    int acc_wide;      // two-word sums (FP64 contexts)
    double rmax;       // largest particle radius
    double inv_tau[2]; // 1/tau_k
    double inv_nu[2];  // 1/nu_k, nu_k = (tau_k - 1/2)/3
    int tau_equal;     // tau_A == tau_B
    ParamsF PF;        // FP32 copies (see ParamsF)
    int* ipos;         // [n][3] floor of the position (FP32 geometry origin)
    float* fsnap;      // [n][9] position - ipos, v(t-1/2), omega(t-1/2) in FP32
    double* red;       // reduction partials
    int red_blocks;
    int dense_psi;     // psi holds rho^k of every fluid node (a full density pass ran this step)
    int dense_mom;     // that pass also wrote j^A + j^B into mom (omega = 1 collision on momenta)
    void* mom;         // [3][pstride] of C: (j^A + j^B)_d of every site, row d
    int sr;            // FP16: stochastic rounding of the stores of the time step
    unsigned sr_key;   // this step's key of the rounding bits
    lb_params P;
};

enum { FLAG_NONFINITE = 1, FLAG_OVERLAP = 2 };
constexpr int PAIR_LIST_MAX = 32;  // listed neighbours per particle

// node codes of the shared-memory planes of the streaming kernels: a fluid
// node, a node beyond a wall, or the index (>= 0) of the particle that owns a
// particle node (the owner map holds -1 on fluid nodes)
constexpr int ND_FLUID = -1, ND_WALL = -2;

// ------------------------------------------------- compensated FP64 sums
struct NSum {
    double s, c;
    __device__ __forceinline__ void add(double x) {
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ void merge(const NSum& o) {
        add(o.s);
        c += o.c;
    }
    __device__ __forceinline__ double value() const { return s + c; }
};

// ----------------------------------------------------------- site helpers
struct SiteNbr {
    int x, y, z;
    int xm, xp, ym, yp, zm, zp;  // wrapped neighbour coordinates
    bool wall_lo, wall_hi;        // z-1 / z+1 lies beyond a wall
};

__device__ __forceinline__ SiteNbr site_nbr(const Lattice& L, int x, int y, int z) {
    SiteNbr n;
    n.x = x; n.y = y; n.z = z;
    n.xm = x == 0 ? L.nx - 1 : x - 1;
    n.xp = x == L.nx - 1 ? 0 : x + 1;
    n.ym = y == 0 ? L.ny - 1 : y - 1;
    n.yp = y == L.ny - 1 ? 0 : y + 1;
    n.zm = z == 0 ? L.nz - 1 : z - 1;
    n.zp = z == L.nz - 1 ? 0 : z + 1;
    n.wall_lo = (z == 0) && !L.per[2];
    n.wall_hi = (z == L.nz - 1) && !L.per[2];
    return n;
}

// site index of the neighbour along link i (caller checks walls first)
__device__ __forceinline__ long long nbr_index(const Lattice& L, const SiteNbr& n, int i) {
    int X = cx(i) == 0 ? n.x : (cx(i) > 0 ? n.xp : n.xm);
    int Y = cy(i) == 0 ? n.y : (cy(i) > 0 ? n.yp : n.ym);
    int Z = cz(i) == 0 ? n.z : (cz(i) > 0 ? n.zp : n.zm);
    return (long long)X + (long long)L.nx * ((long long)Y + (long long)L.ny * Z);
}

__device__ __forceinline__ bool nbr_is_wall(const SiteNbr& n, int i) {
    return (cz(i) < 0 && n.wall_lo) || (cz(i) > 0 && n.wall_hi);
}

// Eq. 5: f_i^eq = w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)   (cs^2 = 1/3)
template <typename C>
__device__ __forceinline__ C feq(int i, C rho, C ux, C uy, C uz, C uu) {
    C cu = C(cx(i)) * ux + C(cy(i)) * uy + C(cz(i)) * uz;
    return wgt<C>(i) * rho * (C(1) + C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu);
}

template <typename S, typename C>
__device__ __forceinline__ C pop_shift(const Lattice& L, int k, int i) {
    return (sizeof(S) == 2) ? wgt<C>(i) * prm<C>(L.P.rho0[k], L.PF.rho0[k]) : C(0);
}

// Load the 2 x 19 populations of one site and form rho^k and j^k
// (Eqs. 6, 7).  The summation order is fixed (i = 0..18) so that every
// kernel obtains bit-identical densities for the same site.
template <int PREC>
__device__ __forceinline__ void load_site(const Lattice& L, const typename Prec<PREC>::S* f,
                                          long long s, typename Prec<PREC>::C (&fv)[2][Q],
                                          typename Prec<PREC>::C (&rho)[2],
                                          typename Prec<PREC>::C (&j)[2][3]) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        C r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            C v = ld_pop(f + pop_index(k * Q + i, s, L.pstride), pop_shift<S, C>(L, k, i));
            fv[k][i] = v;
            r += v;
            if (cx(i) > 0) jx += v; else if (cx(i) < 0) jx -= v;
            if (cy(i) > 0) jy += v; else if (cy(i) < 0) jy -= v;
            if (cz(i) > 0) jz += v; else if (cz(i) < 0) jz -= v;
        }
        rho[k] = r;
        j[k][0] = jx; j[k][1] = jy; j[k][2] = jz;
    }
}

// Eq. 11 (repulsive sign) plus the body force: F^k = -G rho^k sum_i w_i
// psi^kbar(x + c_i) c_i + rho^k g.  psi is rho on fluid nodes, the virtual
// density (Eq. 20) on particle frontier nodes and the wall density beyond a
// wall.
template <typename C>
__device__ __forceinline__ void sc_force(const Lattice& L, const SiteNbr& n, const C (&rho)[2],
                                         C (&F)[2][3]) {
    const C* psi = (const C*)L.psi;
    const C* pw = (const C*)L.psi_wall;
    long long nxy = (long long)L.nx * L.ny;
    C sA[3] = {0, 0, 0}, sB[3] = {0, 0, 0};  // sums of w psi^A c and w psi^B c
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
            pa = __ldg(psi + 2 * m);
            pb = __ldg(psi + 2 * m + 1);
        }
        C w = wgt<C>(i);
        if (cx(i)) { sA[0] += C(cx(i)) * w * pa; sB[0] += C(cx(i)) * w * pb; }
        if (cy(i)) { sA[1] += C(cy(i)) * w * pa; sB[1] += C(cy(i)) * w * pb; }
        if (cz(i)) { sA[2] += C(cz(i)) * w * pa; sB[2] += C(cz(i)) * w * pb; }
    }
    C G = prm<C>(L.P.G, L.PF.G);
#pragma unroll
    for (int d = 0; d < 3; d++) {
        C g = prm<C>(L.P.body_force[d], L.PF.body_force[d]);
        F[0][d] = -G * rho[0] * sB[d] + rho[0] * g;  // component A feels B
        F[1][d] = -G * rho[1] * sA[d] + rho[1] * g;  // component B feels A
    }
}

// Eq. 14 mixture velocity with omega^k = 1/tau_k, and the relaxation
// frequency of the mixture 1/(nubar/cs^2 + 1/2), 1/nubar = sum_k (rho^k/rho)/nu_k.
template <typename C>
__device__ __forceinline__ void mixture(const Lattice& L, const C (&rho)[2], const C (&j)[2][3],
                                        C (&u)[3], C& om) {
    C rt = rho[0] + rho[1];
    if (L.tau_equal) {
        // equal relaxation times: Eq. 14 is sum_k j^k / rho and 1/nubar = 1/nu,
        // so the mixture frequency is exactly 1/tau
        C ir = C(1) / rt;
#pragma unroll
        for (int d = 0; d < 3; d++) u[d] = (j[0][d] + j[1][d]) * ir;
        om = prm<C>(L.inv_tau[0], L.PF.inv_tau[0]);
        return;
    }
    C w0 = prm<C>(L.inv_tau[0], L.PF.inv_tau[0]), w1 = prm<C>(L.inv_tau[1], L.PF.inv_tau[1]);
    C iden = C(1) / (w0 * rho[0] + w1 * rho[1]);
#pragma unroll
    for (int d = 0; d < 3; d++) u[d] = (w0 * j[0][d] + w1 * j[1][d]) * iden;
    C q = (rho[0] * prm<C>(L.inv_nu[0], L.PF.inv_nu[0]) + rho[1] * prm<C>(L.inv_nu[1], L.PF.inv_nu[1])) /
          rt;  // 1/nubar
    om = q / (C(3) + C(0.5) * q);                                     // 1/(3 nubar + 1/2)
}

// U0 = v_p + omega_p x (x - r_p) for a site x next to particle p.  For the
// link along c_i the wall velocity of Eq. 18 is u_w = v_p + omega_p x (r_w -
// r_p) with r_w = x + c_i/2, and c_i . u_w = c_i . U0 because c_i . (omega x
// c_i) = 0: one U0 per site serves every link of that site into p.  The
// offset x - r_p is formed from the integer part of r_p and its fractional
// part, exact in FP64 and accurate to FP32 rounding of a number below 1 in the
// FP32 forms (which read the FP32 particle snapshot).  The loads
// (particle_load) and the arithmetic (particle_u0_of) are split so that a
// caller can issue the loads early.
template <typename C>
struct ParticleRef {
    int ip[3];
    C fr[3], v[3], w[3];
};

template <typename C>
__device__ __forceinline__ ParticleRef<C> particle_load(const Lattice& L, int p) {
    ParticleRef<C> r;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (sizeof(C) == 8) {
            double q = __ldg(L.pos + 3 * p + d);
            r.ip[d] = (int)floor(q);
            r.fr[d] = C(q - (double)r.ip[d]);
            r.v[d] = C(__ldg(L.vel + 3 * p + d));
            r.w[d] = C(__ldg(L.omg + 3 * p + d));
        } else {
            r.ip[d] = __ldg(L.ipos + 3 * p + d);
            r.fr[d] = C(__ldg(L.fsnap + 9 * p + d));
            r.v[d] = C(__ldg(L.fsnap + 9 * p + 3 + d));
            r.w[d] = C(__ldg(L.fsnap + 9 * p + 6 + d));
        }
    }
    return r;
}

template <typename C>
__device__ __forceinline__ void particle_u0_of(const Lattice& L, const ParticleRef<C>& r, int x, int y, int z,
                                               C (&U0)[3], C (&rel)[3]) {
    int xs[3] = {x, y, z}, Ls[3] = {L.nx, L.ny, L.nz};
#pragma unroll
    for (int d = 0; d < 3; d++) {
        int dd = xs[d] - r.ip[d];
        if (L.per[d]) {
            if (2 * dd > Ls[d]) dd -= Ls[d];
            else if (2 * dd < -Ls[d]) dd += Ls[d];
        }
        rel[d] = C(dd) - r.fr[d];
    }
    U0[0] = r.v[0] + (r.w[1] * rel[2] - r.w[2] * rel[1]);
    U0[1] = r.v[1] + (r.w[2] * rel[0] - r.w[0] * rel[2]);
    U0[2] = r.v[2] + (r.w[0] * rel[1] - r.w[1] * rel[0]);
}

template <typename C>
__device__ __forceinline__ void particle_u0(const Lattice& L, int p, int x, int y, int z, C (&U0)[3], C (&rel)[3]) {
    particle_u0_of<C>(L, particle_load<C>(L, p), x, y, z, U0, rel);
}

// Janus wettability of a particle node (Sec. 5.1; App. A wettability angle):
// the switch s in [-1, 1] of the polar angle between d = x - r_p and the
// particle's first body axis, the first column of R(q) (Eq. 31); the node's
// wetting constants are then s zeta^A and -s zeta^B.  s goes from -1 to 1
// across [theta0 - w/2, theta0 + w/2] along the cubic smoothstep.
template <typename C>
__device__ __forceinline__ C janus_switch(const Lattice& L, int p, const C (&d)[3]) {
    const double* q = L.quat + 4 * p;
    const C a = C(q[0]), b = C(q[1]), c = C(q[2]), e = C(q[3]);
    const C n2 = a * a + b * b + c * c + e * e;
    // first column of R(q) for the unnormalised q, divided by |q|^2 below
    const C ax[3] = {a * a + b * b - c * c - e * e, C(2) * (b * c + a * e), C(2) * (b * e - a * c)};
    const C dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (!(dn > C(0))) return C(0);
    C ct = (ax[0] * d[0] + ax[1] * d[1] + ax[2] * d[2]) / (n2 * dn);
    ct = ct > C(1) ? C(1) : (ct < C(-1) ? C(-1) : ct);
    const C th = acos(ct) * C(57.295779513082320876798154814105);  // degrees
    const C th0 = C(L.P.janus_theta0), w = C(L.P.janus_width);
    if (!(w > C(0))) return th < th0 ? C(-1) : C(1);
    C t = (th - (th0 - C(0.5) * w)) / w;
    t = t < C(0) ? C(0) : (t > C(1) ? C(1) : t);
    return C(-1) + C(2) * t * t * (C(3) - C(2) * t);
}

// ---------------------------------------- per-particle fixed-point sums
// The per-particle terms that many threads add to (link forces of Eqs. 19,
// 22-23, the wetting force of Eq. 21, the remap momenta of Eqs. 24-25) are
// summed as fixed-point integers with 64-bit integer atomics, so that a sum
// does not depend on the order in which threads add: it is reproducible bit
// for bit.  Two formats, by the context's precision (L.acc_wide):
//  * FP32 / FP16 contexts: one word, round(v 2^40) (|v| < 2^23, resolution
//    2^-40, far below the FP32 rounding of each term);
//  * FP64 contexts: two words, V = v 2^64 as hi = floor(V / 2^40) and
//    lo = V - hi 2^40 in [0, 2^40] (|v| < 2^39, resolution 2^-64; the lo
//    sums stay below 2^63 for up to 2^23 terms per step); the total is
//    hi 2^-24 + lo 2^-64.
enum { ACC_FLIQ, ACC_TLIQ, ACC_FD, ACC_TD, ACC_FC, ACC_TC, ACC_FS, ACC_TS, ACC_TERMS };

__device__ __forceinline__ unsigned long long* acc_slot(const Lattice& L, int term, int p, int d) {
    return L.acc + (((size_t)term * L.maxc + p) * 3 + d) * 2;
}

// A term outside the range of its format (or not finite) is flagged as a
// non-finite state and not added.
// FP32 terms come from FP32 / FP16 contexts only.
// The words acc_add adds for v (w[1] = 0 in the one-word format); false
// (and the flag raised) if v is out of range.
__device__ __forceinline__ bool acc_words(const Lattice& L, float v, unsigned long long (&w)[2]) {
    if (!(fabsf(v) < 8388608.0f)) {  // 2^23
        atomicOr(L.flags, FLAG_NONFINITE);
        return false;
    }
    w[0] = (unsigned long long)__float2ll_rn(v * 1099511627776.0f);  // 2^40
    w[1] = 0;
    return true;
}

__device__ __forceinline__ bool acc_words(const Lattice& L, double v, unsigned long long (&w)[2]) {
    if (!(fabs(v) < (L.acc_wide ? 549755813888.0 : 8388608.0))) {  // 2^39 / 2^23
        atomicOr(L.flags, FLAG_NONFINITE);
        return false;
    }
    if (!L.acc_wide) {
        w[0] = (unsigned long long)__double2ll_rn(v * 1099511627776.0);
        w[1] = 0;
        return true;
    }
    const double h = floor(v * 16777216.0);           // 2^24
    const double r = v - h * 5.9604644775390625e-08;  // exact, in [0, 2^-24)
    w[0] = (unsigned long long)__double2ll_rn(h);
    w[1] = (unsigned long long)__double2ll_rn(r * 18446744073709551616.0);
    return true;
}

__device__ __forceinline__ void acc_add_words(const Lattice& L, unsigned long long* a,
                                              const unsigned long long (&w)[2]) {
    atomicAdd(a, w[0]);
    if (L.acc_wide) atomicAdd(a + 1, w[1]);
}

__device__ __forceinline__ void acc_add(const Lattice& L, unsigned long long* a, float v) {
    unsigned long long w[2];
    if (acc_words(L, v, w)) atomicAdd(a, w[0]);
}

__device__ __forceinline__ void acc_add(const Lattice& L, unsigned long long* a, double v) {
    unsigned long long w[2];
    if (acc_words(L, v, w)) acc_add_words(L, a, w);
}

__device__ __forceinline__ double acc_value(const Lattice& L, const unsigned long long* a) {
    if (!L.acc_wide) return (double)(long long)a[0] * 9.094947017729282e-13;  // 2^-40
    return (double)(long long)a[0] * 5.9604644775390625e-08 + (double)a[1] * 5.421010862427522e-20;
}

// Neumaier sum in the compute type (per-thread partials before the FP64 merge)
template <typename C>
struct CSum {
    C s, c;
    __device__ __forceinline__ void add(C x) {
        C t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
};

// asynchronous global -> shared copies (cp.async) and their completion
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async_16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ------------------------------------------------ per-device launch state
// The > 48 KB dynamic shared-memory attribute is a property of a function in
// one CUDA context, and the resident-block and SM counts that size the grids
// can differ between devices: each is looked up once per (context, kernel),
// in the context current at the launch.  A context that replaces another on
// the same device (after a device reset) has a new id, so nothing set up in
// the old one is reused.
constexpr int MAX_DEV = 64;

inline int current_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev >= 0 && dev < MAX_DEV ? dev : 0;
}

// Unique id of the calling thread's current CUDA context; 0 when no context
// is current or the driver cannot say (callers then redo their set-up).
unsigned long long current_context_id();

inline int device_sms() {
    static std::atomic<int> sms[MAX_DEV];
    const int dev = current_device();
    int n = sms[dev].load(std::memory_order_relaxed);
    if (!n) {
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        n = n > 0 ? n : 1;
        sms[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

// Allow `smem` bytes of dynamic shared memory for kernel FN in the current
// context (once) and return its resident blocks per SM at `threads` threads.
template <auto FN>
inline int kernel_setup(int threads, size_t smem) {
    static std::atomic<unsigned long long> ctx[MAX_DEV];
    static std::atomic<int> per_sm[MAX_DEV];
    const int dev = current_device();
    const unsigned long long id = current_context_id();
    if (id && ctx[dev].load(std::memory_order_acquire) == id) return per_sm[dev].load(std::memory_order_relaxed);
    // the opt-in beyond 48 KB counts the kernel's static shared memory too
    cudaFuncAttributes fa;
    const size_t stat = cudaFuncGetAttributes(&fa, FN) == cudaSuccess ? fa.sharedSizeBytes : 0;
    if (smem + stat > 48 * 1024) cudaFuncSetAttribute(FN, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, FN, threads, smem);
    n = n > 0 ? n : 1;
    per_sm[dev].store(n, std::memory_order_relaxed);
    ctx[dev].store(id, std::memory_order_release);
    return n;
}

// kernel launchers (each returns the number of kernels it launched)
int launch_init_fields(const Lattice& L, int prec, const double* stage, cudaStream_t st);
int launch_fluid_step(const Lattice& L, int prec, cudaStream_t st);
// the one-component fluid (lbgb_single.cu)
int launch_single_init(const Lattice& L, int prec, const double* stage, cudaStream_t st);
int launch_single_step(const Lattice& L, int prec, cudaStream_t st);
int launch_single_face_values(const Lattice& L, int prec, cudaStream_t st);
int launch_single_fields_out(const Lattice& L, int prec, double* stage, cudaStream_t st);
int launch_single_totals_partial(const Lattice& L, int prec, cudaStream_t st);
int launch_single_populations_out(const Lattice& L, int prec, int i, double* stage, cudaStream_t st);
// the links across the z faces after the lean push (with particles and
// tau^A = tau^B = 1)
int launch_wall_bounce(const Lattice& L, int prec, cudaStream_t st);
int launch_shell_density(const Lattice& L, int prec, cudaStream_t st);
int launch_density(const Lattice& L, int prec, cudaStream_t st);
int launch_wall_psi(const Lattice& L, int prec, cudaStream_t st);
int launch_face_values(const Lattice& L, int prec, cudaStream_t st);
int launch_fields_out(const Lattice& L, int prec, double* stage, cudaStream_t st);
int launch_totals(const Lattice& L, int prec, double* out_dev, cudaStream_t st);
int launch_populations_out(const Lattice& L, int prec, int k, int i, double* stage, cudaStream_t st);
int launch_clear_map(const Lattice& L, cudaStream_t st);

int launch_map_initial(const Lattice& L, int prec, int first, int count, cudaStream_t st);
// the link classes nb: of every site (full), or around the nodes the remap
// of this step listed
int launch_link_classes(const Lattice& L, bool full, cudaStream_t st);
int launch_remap(const Lattice& L, int prec, int maxc, cudaStream_t st);
int launch_virtual(const Lattice& L, int prec, int store_terms, cudaStream_t st);
// Eqs. 26-27 and the side walls into Fpair (reads positions and velocities only)
int launch_pairs(const Lattice& L, void* cells, size_t cell_cap, bool force_build, cudaStream_t st);
// Eqs. 28-35: totals, leap-frog, quaternions, snapshot
int launch_integrate(const Lattice& L, cudaStream_t st);
int launch_snapshot(const Lattice& L, cudaStream_t st);

size_t adjoint_field_bytes(const Lattice& L, int prec);
size_t adjoint_scratch_bytes(const Lattice& L, int prec);
int launch_adjoint_step(const Lattice& L, int prec, const void* in, void* out, void* scratch,
                        const double* dJdF_dev, double* grads_dev, cudaStream_t st);
int launch_adjoint_seed(const Lattice& L, int prec, void* adj, void* scratch, double weight, double* value_dev,
                        cudaStream_t st);
int launch_adjoint_initial(const Lattice& L, int prec, const void* adj, double* grad, cudaStream_t st);
int launch_drag_gradient(int n, const double* F, double weight, double eps, double* out, cudaStream_t st);

}  // namespace lbgb
