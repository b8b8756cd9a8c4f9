// lbgb_api.cu -- host side of the C ABI declared in include/lbgb.h:
// argument validation, workspace carving, the per-step launch sequence and
// the host<->device copies of the read-out calls.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cuda.h>
#include <stdlib.h>

#include <mutex>
#include <new>

#include "lbgb_internal.cuh"

using namespace lbgb;

// The driver's context queries, found through the runtime so that the library
// links against the runtime only.
unsigned long long lbgb::current_context_id() {
    typedef CUresult (*GetCurrent)(CUcontext*);
    typedef CUresult (*GetId)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (GetCurrent)p;
        p = nullptr;
        q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (GetId)p;
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c) return 0;
    if (get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

struct lb_ctx {
    Lattice L;
    int prec;
    int maxc;
    cudaStream_t stream;
    // the pair forces depend only on the particle state of the previous step:
    // they run on `side` (created by the library, high priority) while the
    // lattice kernels run on `stream`; the integrator waits for them
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
    char* ws;
    size_t ws_bytes;
    int have_params, have_fields, stepped;
    int all_fixed;              // every particle immobile (infinite mass, at rest)
    long long launches;
    double* totals_dev;
    void* cells;
    size_t cells_bytes;
    int prof_on;
    int prof_n[LB_KERNEL_KINDS];           // recorded event pairs, by kernel (LB_KERNEL_*)
    cudaEvent_t* prof_ev[LB_KERNEL_KINDS]; // 2 * PROF_MAX events each, created on first use
    char* rec_states;           // lb_record: f(t) of each recorded step, or null
    double* rec_forces;         // lb_record: F_liq after each recorded step, or null
    int rec_left, rec_i;        // steps still to record, steps recorded
    unsigned long long sr_seed; // stochastic rounding: seed, and steps taken with it
    unsigned long long sr_step;
    int vl_valid;               // the particle pair list holds the current particles
    int nb_valid;               // the link classes match the node map up to this step's remap
    char err[512];
};

namespace {

const size_t ALIGN = 256;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

size_t storage_bytes(int prec) { return prec == LB_FP64 ? 8 : (prec == LB_FP32 ? 4 : 2); }
size_t compute_bytes(int prec) { return prec == LB_FP64 ? 8 : 4; }
// bytes of one population state (both buffers have this size)
size_t state_bytes(const lb_ctx* ctx) {
    return (size_t)ctx->L.ncomp * Q * ctx->L.pstride * storage_bytes(ctx->prec);
}

const int DOUBLES_PER_PARTICLE = 57;  // pos..Ttot, see carve()
// seed of the default stochastic rounding of FP16 contexts (any constant: the
// sequence of rounding bits is fixed by it and the steps since lb_init_fields)
const unsigned long long SR_DEFAULT_SEED = 0x2545F4914F6CDD1Dull;
const int RED_BLOCKS = 1024;
const int PROF_MAX = 16384;

struct Layout {
    size_t f0, f1, mom, psi, psi_wall, face, mask, owner, evt, nb, nb_chg, flags, col, prev, acc, vl, ipos, fsnap, cells,
        cells_bytes, red, totals, total;
    long long pstride;
};

// ncomp = 1: the one-component fluid holds one population per link and
// site and none of the per-site arrays of the particle coupling
Layout layout(int nx, int ny, int nz, int prec, int maxc, int ncomp) {
    Layout l;
    long long N = (long long)nx * ny * nz;
    // population planes: pstride component pairs (one component: single
    // elements) each, SKEW of padding at both ends (pop_index, pop1_index)
    l.pstride = (N + 2 * SKEW + 63) / 64 * 64;
    size_t off = 0;
    size_t fb = (size_t)ncomp * Q * l.pstride * storage_bytes(prec);
    const long long Np = ncomp == 2 ? N : 0;  // per-site arrays of the coupled lattice
    // the second population buffer doubles as the FP64 staging area of the
    // read-out calls (5 doubles per site), so it is at least that large
    size_t fb1 = fb > (size_t)5 * N * 8 ? fb : (size_t)5 * N * 8;
    l.f0 = off; off = align_up(off + fb);
    l.f1 = off; off = align_up(off + fb1);
    l.mom = off; off = align_up(off + (size_t)3 * (ncomp == 2 ? l.pstride : 0) * compute_bytes(prec));
    l.psi = off; off = align_up(off + (size_t)2 * Np * compute_bytes(prec));
    l.psi_wall = off; off = align_up(off + (size_t)4 * nx * ny * compute_bytes(prec));
    l.face = off; off = align_up(off + (size_t)10 * nx * ny * compute_bytes(prec));
    l.mask = off; off = align_up(off + (size_t)Np);
    l.owner = off; off = align_up(off + (size_t)Np * 4);
    l.evt = off; off = align_up(off + (size_t)Np * 4);
    l.nb = off; off = align_up(off + (size_t)Np * 4);
    l.nb_chg = off; off = align_up(off + (size_t)(ncomp == 2 ? 8 + NB_CHG_CAP : 0) * 4);
    l.flags = off; off = align_up(off + 64);
    int mc = maxc > 0 ? maxc : 1;
    l.col = off; off = align_up(off + (size_t)mc * DOUBLES_PER_PARTICLE * 8);
    l.prev = off; off = align_up(off + (size_t)mc * 4);
    l.acc = off; off = align_up(off + (size_t)ACC_TERMS * mc * 6 * 8);
    // pair list: positions at the build (FP64), builds counter, flag,
    // counts, neighbours
    l.vl = off; off = align_up(off + (size_t)mc * 24 + 16 + (size_t)mc * 4 * (1 + PAIR_LIST_MAX));
    l.ipos = off; off = align_up(off + (size_t)mc * 12);
    l.fsnap = off; off = align_up(off + (size_t)mc * 36);
    // particle cell list: counts and starts of up to 64^3 cells, then the items
    l.cells_bytes = ncomp == 2 ? ((size_t)2 * 64 * 64 * 64 + 1 + (size_t)mc) * 4 : 0;
    l.cells = off; off = align_up(off + l.cells_bytes);
    l.red = off; off = align_up(off + (size_t)RED_BLOCKS * 16 * 8);
    l.totals = off; off = align_up(off + 8 * 8);
    l.total = off;
    return l;
}

int set_err(lb_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_check(lb_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return LB_OK;
    return set_err(c, LB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        int rc_ = cuda_check(ctx, (call), what);         \
        if (rc_) return rc_;                             \
    } while (0)

// the start (end = 0) or end (end = 1) event of one timed launch of a kernel
// kind, while profiling is on and the record has room
static int prof_mark(lb_ctx* ctx, int kind, int end, cudaStream_t s) {
    if (!ctx->prof_on || ctx->prof_n[kind] >= PROF_MAX) return LB_OK;
    CK(cudaEventRecord(ctx->prof_ev[kind][2 * ctx->prof_n[kind] + end], s), "profile event");
    ctx->prof_n[kind] += end;
    return LB_OK;
}

int launched(lb_ctx* ctx, int n, const char* what) {
    ctx->launches += n;
    return cuda_check(ctx, cudaGetLastError(), what);
}

double* stage_ptr(lb_ctx* ctx) { return (double*)ctx->L.f_nxt; }

}  // namespace

extern "C" {

static const long long MAX_SITES = (1LL << 31) - 4096;

// the precision code and the number of components of a prec argument
static bool split_prec(int& prec, int& ncomp, int max_colloids) {
    ncomp = (prec & LB_ONE_COMPONENT) ? 1 : 2;
    prec &= ~LB_ONE_COMPONENT;
    if (prec != LB_FP64 && prec != LB_FP32 && prec != LB_FP16) return false;
    return ncomp == 2 || max_colloids == 0;  // one component: no particles
}

int lb_workspace_bytes(int nx, int ny, int nz, int prec, int max_colloids, size_t* bytes) {
    if (!bytes || nx < 4 || ny < 4 || nz < 4 || max_colloids < 0) return LB_ERR_ARG;
    int ncomp;
    if (!split_prec(prec, ncomp, max_colloids)) return LB_ERR_ARG;
    *bytes = layout(nx, ny, nz, prec, max_colloids, ncomp).total;
    return LB_OK;
}

static cudaError_t create_side_stream(lb_ctx* ctx) {
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
    return e;
}

static void destroy_side_stream(lb_ctx* ctx) {
    if (ctx->side) {
        cudaStreamSynchronize(ctx->side);
        cudaStreamDestroy(ctx->side);
    }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    ctx->side = NULL;
    ctx->ev_fork = ctx->ev_join = NULL;
}

int lb_create(int nx, int ny, int nz, int prec, int max_colloids, void* d_workspace, size_t bytes,
              void* cuda_stream, lb_ctx** out) {
    if (!out) return LB_ERR_ARG;
    *out = NULL;
    if (nx < 4 || ny < 4 || nz < 4 || (nx % 4) != 0 || max_colloids < 0) return LB_ERR_ARG;
    int ncomp;
    if (!split_prec(prec, ncomp, max_colloids)) return LB_ERR_ARG;
    // the lattice kernels index sites with 32-bit integers
    if ((long long)nx * ny * nz > MAX_SITES) return LB_ERR_ARG;
    if (!d_workspace || ((uintptr_t)d_workspace % ALIGN) != 0) return LB_ERR_ARG;
    Layout l = layout(nx, ny, nz, prec, max_colloids, ncomp);
    if (bytes < l.total) return LB_ERR_NOMEM;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, d_workspace) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return LB_ERR_ARG;
    }
    lb_ctx* ctx = new (std::nothrow) lb_ctx;
    if (!ctx) return LB_ERR_NOMEM;
    memset(ctx, 0, sizeof(*ctx));
    ctx->prec = prec;
    ctx->maxc = max_colloids;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->ws = (char*)d_workspace;
    ctx->ws_bytes = bytes;
    Lattice& L = ctx->L;
    L.nx = nx; L.ny = ny; L.nz = nz;
    L.N = (long long)nx * ny * nz;
    L.ncomp = ncomp;
    L.pstride = l.pstride;
    L.per[0] = L.per[1] = L.per[2] = 1;
    L.f_cur = ctx->ws + l.f0;
    L.f_nxt = ctx->ws + l.f1;
    L.mom = ctx->ws + l.mom;
    L.psi = ctx->ws + l.psi;
    L.psi_wall = ctx->ws + l.psi_wall;
    L.face = ctx->ws + l.face;
    L.mask = (uint8_t*)(ctx->ws + l.mask);
    L.owner = (int*)(ctx->ws + l.owner);
    L.evt = (int*)(ctx->ws + l.evt);
    L.nb = (uint32_t*)(ctx->ws + l.nb);
    L.nb_chg = (int*)(ctx->ws + l.nb_chg);
    L.flags = (int*)(ctx->ws + l.flags);
    int mc = max_colloids > 0 ? max_colloids : 1;
    double* c = (double*)(ctx->ws + l.col);
    double** slots3[] = {&L.pos, &L.vel, &L.omg};
    for (int a = 0; a < 3; a++) { *slots3[a] = c; c += 3 * mc; }
    L.quat = c; c += 4 * mc;
    L.rad = c; c += mc;
    L.mass = c; c += mc;
    double** more[] = {&L.Fliq, &L.Tliq, &L.Fliq_prev, &L.Tliq_prev, &L.Fd, &L.Td, &L.Fc,
                       &L.Tc, &L.Fs, &L.Ts, &L.Fpair, &L.Ftot, &L.Ttot};
    for (int a = 0; a < 13; a++) { *more[a] = c; c += 3 * mc; }
    L.prev_valid = (int*)(ctx->ws + l.prev);
    L.acc = (unsigned long long*)(ctx->ws + l.acc);
    L.vl_ref = (double*)(ctx->ws + l.vl);
    L.vl_builds = (unsigned long long*)(L.vl_ref + 3 * mc);
    L.vl_flag = (int*)(L.vl_builds + 1);
    L.vl_cnt = L.vl_flag + 2;
    L.vl_nb = L.vl_cnt + mc;
    L.maxc = mc;
    L.acc_wide = prec == LB_FP64;
    L.ipos = (int*)(ctx->ws + l.ipos);
    L.fsnap = (float*)(ctx->ws + l.fsnap);
    L.red = (double*)(ctx->ws + l.red);
    L.red_blocks = RED_BLOCKS;
    ctx->totals_dev = (double*)(ctx->ws + l.totals);
    ctx->cells = ctx->ws + l.cells;
    ctx->cells_bytes = l.cells_bytes;
    L.nc = 0;
    // FP16 storage rounds stochastically by default (lb_set_rounding)
    L.sr = prec == LB_FP16;
    ctx->sr_seed = SR_DEFAULT_SEED;
    ctx->sr_step = 0;
    // empty node map, no particles, no error flags (the per-site arrays of
    // the coupling exist on the two-component lattice only: sizes of layout())
    const size_t Np = ncomp == 2 ? (size_t)L.N : 0;
    cudaError_t e = cudaMemsetAsync(ctx->ws + l.mask, 0, Np, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ws + l.owner, 0xff, Np * 4, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ws + l.evt, 0, Np * 4, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ws + l.flags, 0, 64, ctx->stream);
    // psi: kernels read it on particle nodes that no virtual density has
    // reached yet (deep nodes), where any finite value serves
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ws + l.psi, 0, 2 * Np * compute_bytes(prec), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ws + l.col, 0, (size_t)mc * DOUBLES_PER_PARTICLE * 8, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ws + l.prev, 0, (size_t)mc * 4, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ws + l.vl, 0, (size_t)mc * 24 + 16, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = create_side_stream(ctx);
    if (e != cudaSuccess) {
        destroy_side_stream(ctx);
        delete ctx;
        return LB_ERR_CUDA;
    }
    *out = ctx;
    return LB_OK;
}

int lb_set_params(lb_ctx* ctx, const lb_params* p) {
    if (!ctx || !p) return LB_ERR_ARG;
    if (!(p->tau[0] > 0.5) || !(p->tau[1] > 0.5) || !isfinite(p->tau[0]) || !isfinite(p->tau[1]))
        return set_err(ctx, LB_ERR_ARG, "tau must be finite and > 1/2");
    if (p->bc[0] != 1 || p->bc[1] != 1 || (p->bc[2] != 0 && p->bc[2] != 1))
        return set_err(ctx, LB_ERR_ARG, "walls are supported only along z (bc = {1,1,0|1})");
    const double* vals[] = {&p->G, &p->zeta[0], &p->zeta[1], &p->rho0[0], &p->rho0[1], &p->hertz_K,
                            &p->hertz_sigma, &p->hertz_rcap, &p->side_wall_k, &p->side_wall_d};
    for (unsigned a = 0; a < sizeof(vals) / sizeof(vals[0]); a++)
        if (!isfinite(*vals[a])) return set_err(ctx, LB_ERR_ARG, "non-finite parameter");
    for (int d = 0; d < 3; d++)
        if (!isfinite(p->wall_u_lo[d]) || !isfinite(p->wall_u_hi[d]) || !isfinite(p->body_force[d]))
            return set_err(ctx, LB_ERR_ARG, "non-finite wall velocity or body force");
    if (p->lub_on && !(p->lub_hmin > 0.0 && p->lub_hn > p->lub_hmin))
        return set_err(ctx, LB_ERR_ARG, "lubrication needs 0 < lub_hmin < lub_hn");
    if (p->janus && !(isfinite(p->janus_theta0) && isfinite(p->janus_width) && p->janus_width >= 0.0))
        return set_err(ctx, LB_ERR_ARG, "janus needs a finite switch angle and a width >= 0");
    if (!(p->rcut >= 0.0 && isfinite(p->rcut) && p->delr >= 0.0 && isfinite(p->delr)))
        return set_err(ctx, LB_ERR_ARG, "rcut and delr must be finite and >= 0");
    for (int f = 0; f < 2; f++) {
        if (p->open[f] < 0 || p->open[f] > 3) return set_err(ctx, LB_ERR_ARG, "open face types are 0..3");
        if (ctx->L.ncomp == 1 && (p->open[f] == 1 || p->open[f] == 3))
            return set_err(ctx, LB_ERR_ARG, "the one-component lattice has wall and velocity faces only");
        if (p->open[f] != 0 && p->bc[2] != 0)
            return set_err(ctx, LB_ERR_ARG, "open faces need bc[2] = 0 (the z faces)");
        for (int k = 0; k < 2; k++)
            if (!(p->open_rho[f][k] >= 0.0 && isfinite(p->open_rho[f][k])))
                return set_err(ctx, LB_ERR_ARG, "open face densities must be finite and >= 0");
    }
    if (p->open_extrap != 0 && p->open_extrap != 1) return set_err(ctx, LB_ERR_ARG, "open_extrap is 0 or 1");
    if (ctx->stepped && p->bc[2] != ctx->L.P.bc[2])
        return set_err(ctx, LB_ERR_STATE, "boundary conditions cannot change after stepping");
    ctx->L.P = *p;
    ctx->vl_valid = 0;
    ParamsF& f = ctx->L.PF;
    for (int k = 0; k < 2; k++) {
        ctx->L.inv_tau[k] = 1.0 / p->tau[k];
        ctx->L.inv_nu[k] = 3.0 / (p->tau[k] - 0.5);
        f.inv_tau[k] = (float)ctx->L.inv_tau[k];
        f.inv_nu[k] = (float)ctx->L.inv_nu[k];
        f.rho0[k] = (float)p->rho0[k];
    }
    ctx->L.tau_equal = p->tau[0] == p->tau[1];
    f.G = (float)p->G;
    for (int d = 0; d < 3; d++) {
        f.body_force[d] = (float)p->body_force[d];
        f.wall_u_lo[d] = (float)p->wall_u_lo[d];
        f.wall_u_hi[d] = (float)p->wall_u_hi[d];
    }
    ctx->L.per[0] = 1;
    ctx->L.per[1] = 1;
    ctx->L.per[2] = p->bc[2];
    ctx->have_params = 1;
    return LB_OK;
}

int lb_init_fields(lb_ctx* ctx, const double* rhoA, const double* rhoB, const double* u) {
    if (!ctx || !rhoA || (!rhoB && ctx->L.ncomp == 2)) return LB_ERR_ARG;
    if (!ctx->have_params) return set_err(ctx, LB_ERR_STATE, "lb_set_params must come first");
    Lattice& L = ctx->L;
    size_t nb = (size_t)L.N * 8;
    double* st = stage_ptr(ctx);
    CK(cudaMemcpyAsync(st, rhoA, nb, cudaMemcpyHostToDevice, ctx->stream), "copy rhoA");
    if (L.ncomp == 2) CK(cudaMemcpyAsync(st + L.N, rhoB, nb, cudaMemcpyHostToDevice, ctx->stream), "copy rhoB");
    if (u) CK(cudaMemcpyAsync(st + 2 * L.N, u, 3 * nb, cudaMemcpyHostToDevice, ctx->stream), "copy u");
    else CK(cudaMemsetAsync(st + 2 * L.N, 0, 3 * nb, ctx->stream), "zero u");
    L.nc = 0;
    ctx->all_fixed = 1;
    ctx->sr_step = 0;  // a new state starts the rounding sequence afresh
    ctx->nb_valid = 0;
    int n = 0;
    if (L.ncomp == 1) {
        n += launch_single_init(L, ctx->prec, st, ctx->stream);
    } else {
        n += launch_clear_map(L, ctx->stream);
        n += launch_init_fields(L, ctx->prec, st, ctx->stream);
    }
    int rc = launched(ctx, n, "init kernels");
    if (rc) return rc;
    CK(cudaStreamSynchronize(ctx->stream), "init sync");
    ctx->have_fields = 1;
    ctx->stepped = 0;
    return LB_OK;
}

int lb_add_colloids(lb_ctx* ctx, int n, const double* pos, const double* vel, const double* omega,
                    const double* quat, const double* radius, const double* mass) {
    if (!ctx || n < 0 || (n > 0 && (!pos || !radius || !mass))) return LB_ERR_ARG;
    if (!ctx->have_fields) return set_err(ctx, LB_ERR_STATE, "lb_init_fields must come first");
    if (n > 0 && ctx->L.ncomp == 1) return set_err(ctx, LB_ERR_ARG, "a one-component lattice holds no particles");
    if (ctx->stepped) return set_err(ctx, LB_ERR_STATE, "particles must be added before the first step");
    Lattice& L = ctx->L;
    if (L.nc + n > ctx->maxc) return set_err(ctx, LB_ERR_STATE, "more than max_colloids particles");
    if (n == 0) return LB_OK;
    int Ls[3] = {L.nx, L.ny, L.nz};
    double* h = new (std::nothrow) double[(size_t)n * 17];
    if (!h) return LB_ERR_NOMEM;
    double *hp = h, *hv = h + 3 * n, *hw = h + 6 * n, *hq = h + 9 * n, *hr = h + 13 * n, *hm = h + 14 * n;
    double rmax = L.rmax;
    for (int p = 0; p < n; p++) {
        double R = radius[p];
        if (!(R > 0.0) || !isfinite(R) || !(mass[p] > 0.0) || isnan(mass[p])) {
            delete[] h;
            return set_err(ctx, LB_ERR_ARG, "particle %d: radius must be finite > 0, mass > 0", p);
        }
        for (int d = 0; d < 3; d++) {
            double x = pos[3 * p + d];
            if (!isfinite(x)) { delete[] h; return set_err(ctx, LB_ERR_ARG, "non-finite position"); }
            if (L.per[d]) {
                if (2.0 * R + 5.0 >= (double)Ls[d]) {
                    delete[] h;
                    return set_err(ctx, LB_ERR_ARG, "particle %d too large for the box", p);
                }
                x = x - (double)Ls[d] * floor(x / (double)Ls[d]);
            } else if (x < 0.0 || x > (double)Ls[d] - 1.0) {
                delete[] h;
                return set_err(ctx, LB_ERR_ARG, "particle %d outside the walls", p);
            }
            hp[3 * p + d] = x;
            hv[3 * p + d] = vel ? vel[3 * p + d] : 0.0;
            hw[3 * p + d] = omega ? omega[3 * p + d] : 0.0;
        }
        for (int d = 0; d < 4; d++) hq[4 * p + d] = quat ? quat[4 * p + d] : (d == 0 ? 1.0 : 0.0);
        hr[p] = R;
        hm[p] = mass[p];
        if (R > rmax) rmax = R;
    }
    int first = L.nc;
    cudaStream_t s = ctx->stream;
    int fixed = first == 0 ? 1 : ctx->all_fixed;
    for (int p = 0; p < n; p++) {
        if (!isinf(hm[p])) fixed = 0;
        for (int d = 0; d < 3; d++)
            if (hv[3 * p + d] != 0.0 || hw[3 * p + d] != 0.0) fixed = 0;
    }
    cudaError_t e = cudaMemcpyAsync(L.pos + 3 * first, hp, 24 * (size_t)n, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(L.vel + 3 * first, hv, 24 * (size_t)n, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(L.omg + 3 * first, hw, 24 * (size_t)n, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(L.quat + 4 * first, hq, 32 * (size_t)n, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(L.rad + first, hr, 8 * (size_t)n, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(L.mass + first, hm, 8 * (size_t)n, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemsetAsync(L.prev_valid + first, 0, 4 * (size_t)n, s);
    if (!e) e = cudaMemsetAsync(L.flags, 0, 4, s);
    if (!e) e = cudaStreamSynchronize(s);
    delete[] h;
    if (e) return cuda_check(ctx, e, "copy particles");
    L.nc = first + n;
    L.rmax = rmax;
    ctx->all_fixed = fixed;
    ctx->vl_valid = 0;
    ctx->nb_valid = 0;
    // the FP32 snapshot first: the map kernel of the FP32 forms reads it
    int nl = launch_snapshot(L, s);
    nl += launch_map_initial(L, ctx->prec, first, n, s);
    int rc = launched(ctx, nl, "map kernel");
    if (rc) return rc;
    int flags = 0;
    CK(cudaMemcpyAsync(&flags, L.flags, 4, cudaMemcpyDeviceToHost, s), "read flags");
    CK(cudaStreamSynchronize(s), "map sync");
    if (flags & FLAG_OVERLAP) return set_err(ctx, LB_ERR_OVERLAP, "particles overlap on the lattice");
    return LB_OK;
}

// key of the stochastic-rounding bits of step t: the SplitMix64 finaliser
// (Steele, Lea, Flood) of seed + t, folded to 32 bits
static unsigned sr_key(unsigned long long seed, unsigned long long t) {
    unsigned long long z = seed + (t + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (unsigned)(z ^ (z >> 32));
}

int lb_set_rounding(lb_ctx* ctx, int mode, unsigned long long seed) {
    if (!ctx) return LB_ERR_ARG;
    if (mode != LB_ROUND_NEAREST && mode != LB_ROUND_STOCHASTIC) return set_err(ctx, LB_ERR_ARG, "unknown rounding mode");
    ctx->L.sr = mode == LB_ROUND_STOCHASTIC && ctx->prec == LB_FP16;
    ctx->sr_seed = seed;
    ctx->sr_step = 0;
    return LB_OK;
}

// the link classes (NB_*) of every site, when they are not kept up to date
static int ensure_link_classes(lb_ctx* ctx, cudaStream_t st) {
    if (ctx->nb_valid) return 0;
    ctx->nb_valid = 1;
    return launch_link_classes(ctx->L, true, st);
}

int lb_step(lb_ctx* ctx, int nsteps) {
    if (!ctx || nsteps < 0) return LB_ERR_ARG;
    if (!ctx->have_fields) return set_err(ctx, LB_ERR_STATE, "lb_init_fields must come first");
    Lattice& L = ctx->L;
    cudaStream_t s = ctx->stream;
    CK(cudaMemsetAsync(L.flags, 0, 4, s), "clear flags");
    for (int t = 0; L.ncomp == 1 && t < nsteps; t++) {
        // the one-component fluid: one kernel per step (Eqs. 5-7, 16, 3, 9)
        if (L.sr) L.sr_key = sr_key(ctx->sr_seed, ctx->sr_step++);
        const int n0 = launch_single_face_values(L, ctx->prec, s);  // extrapolated face densities
        if (int rc = prof_mark(ctx, LB_KERNEL_FUSED, 0, s)) return rc;
        const int n = n0 + launch_single_step(L, ctx->prec, s);
        if (int rc = prof_mark(ctx, LB_KERNEL_FUSED, 1, s)) return rc;
        if (int rc = launched(ctx, n, "step kernel")) return rc;
        void* tmp = L.f_cur;
        L.f_cur = L.f_nxt;
        L.f_nxt = tmp;
        ctx->stepped = 1;
    }
    for (int t = 0; L.ncomp == 2 && t < nsteps; t++) {
        int n = 0;
        const bool rec = ctx->rec_left > 0;
        if (rec && ctx->rec_states)
            CK(cudaMemcpyAsync(ctx->rec_states + (size_t)ctx->rec_i * state_bytes(ctx), L.f_cur, state_bytes(ctx),
                               cudaMemcpyDeviceToDevice, s),
               "record state");
        if (L.nc > 0) {  // Eqs. 26, 27 on the side stream, from r(t), v(t - 1/2)
            CK(cudaEventRecord(ctx->ev_fork, s), "fork event");
            CK(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0), "fork wait");
            n += launch_pairs(L, ctx->cells, ctx->cells_bytes, !ctx->vl_valid, ctx->side);
            ctx->vl_valid = 1;
            CK(cudaEventRecord(ctx->ev_join, ctx->side), "join event");
        }
        if (L.sr) L.sr_key = sr_key(ctx->sr_seed, ctx->sr_step++);
        n += launch_remap(L, ctx->prec, ctx->maxc, s);  // destroy / create (Eqs. 24, 25)
        const bool unit = L.P.tau[0] == 1.0 && L.P.tau[1] == 1.0;
        if (L.nc > 0) {
            n += launch_link_classes(L, !ctx->nb_valid, s);
            ctx->nb_valid = 1;
        } else if (unit) {
            n += ensure_link_classes(ctx, s);  // no particles: every word 0, once
        }
        // rho^k (Eq. 6) of every fluid node when particles need virtual
        // densities (Eq. 20) or omega = 1; with omega = 1 the pass also
        // writes j^k, and the lean kernel collides from the moments instead of
        // re-reading the populations.  Otherwise (no particles, other tau)
        // only the planes next to the walls (the plain fused kernel then forms
        // its halo densities itself).
        L.dense_psi = L.nc > 0 || unit;
        L.dense_mom = L.dense_psi && unit;
        if (L.dense_psi) {
            if (int rc = prof_mark(ctx, LB_KERNEL_DENSITY, 0, s)) return rc;
            n += launch_density(L, ctx->prec, s);
            if (int rc = prof_mark(ctx, LB_KERNEL_DENSITY, 1, s)) return rc;
        } else {
            n += launch_shell_density(L, ctx->prec, s);
        }
        n += launch_wall_psi(L, ctx->prec, s);         // wall densities
        n += launch_face_values(L, ctx->prec, s);      // extrapolated open-face values (Sec. 2.2)
        n += launch_virtual(L, ctx->prec, 1, s);       // Eqs. 20, 21
        if (int rc = prof_mark(ctx, LB_KERNEL_FUSED, 0, s)) return rc;
        // Eqs. 11, 14, 16, 3, 9, 17; the link forces of Eqs. 19, 22, 23
        n += launch_fluid_step(L, ctx->prec, s);
        if (int rc = prof_mark(ctx, LB_KERNEL_FUSED, 1, s)) return rc;
        if (L.nc > 0) CK(cudaStreamWaitEvent(s, ctx->ev_join, 0), "join wait");
        n += launch_integrate(L, s);  // Eqs. 28-35
        int rc = launched(ctx, n, "step kernels");
        if (rc) return rc;
        void* tmp = L.f_cur;
        L.f_cur = L.f_nxt;
        L.f_nxt = tmp;
        ctx->stepped = 1;
        if (rec) {
            if (ctx->rec_forces && L.nc > 0)
                CK(cudaMemcpyAsync(ctx->rec_forces + (size_t)ctx->rec_i * L.nc * 3, L.Fliq, (size_t)L.nc * 24,
                                   cudaMemcpyDeviceToDevice, s),
                   "record forces");
            ctx->rec_i++;
            ctx->rec_left--;
        }
    }
    int flags = 0;
    CK(cudaMemcpyAsync(&flags, L.flags, 4, cudaMemcpyDeviceToHost, s), "read flags");
    CK(cudaStreamSynchronize(s), "step sync");
    if (flags & FLAG_OVERLAP) return set_err(ctx, LB_ERR_OVERLAP, "two particles claimed one node");
    if (flags & FLAG_NONFINITE) return set_err(ctx, LB_ERR_NONFINITE, "non-finite or negative density");
    return LB_OK;
}

// density, wetting and wall fields of the current state (no particle terms)
// the virtual densities find the frontier nodes by the link classes: rebuild
// them if the node map changed outside lb_step (number of launches)

static int current_forces(lb_ctx* ctx) {
    Lattice& L = ctx->L;
    if (L.ncomp == 1) return LB_OK;  // no Shan-Chen or particle terms
    int n = ensure_link_classes(ctx, ctx->stream);
    n += launch_density(L, ctx->prec, ctx->stream);
    n += launch_wall_psi(L, ctx->prec, ctx->stream);
    n += launch_virtual(L, ctx->prec, 0, ctx->stream);
    return launched(ctx, n, "density kernels");
}

int lb_get_fields(lb_ctx* ctx, double* rhoA, double* rhoB, double* u) {
    if (!ctx) return LB_ERR_ARG;
    if (!ctx->have_fields) return set_err(ctx, LB_ERR_STATE, "no fields");
    Lattice& L = ctx->L;
    int rc = current_forces(ctx);
    if (rc) return rc;
    double* st = stage_ptr(ctx);
    rc = launched(ctx, L.ncomp == 1 ? launch_single_fields_out(L, ctx->prec, st, ctx->stream)
                                    : launch_fields_out(L, ctx->prec, st, ctx->stream),
                  "fields kernel");
    if (rc) return rc;
    size_t nb = (size_t)L.N * 8;
    if (rhoA) CK(cudaMemcpyAsync(rhoA, st, nb, cudaMemcpyDeviceToHost, ctx->stream), "copy rhoA");
    if (rhoB) CK(cudaMemcpyAsync(rhoB, st + L.N, nb, cudaMemcpyDeviceToHost, ctx->stream), "copy rhoB");
    if (u) CK(cudaMemcpyAsync(u, st + 2 * L.N, 3 * nb, cudaMemcpyDeviceToHost, ctx->stream), "copy u");
    CK(cudaStreamSynchronize(ctx->stream), "fields sync");
    return LB_OK;
}

int lb_get_totals(lb_ctx* ctx, double* out) {
    if (!ctx || !out) return LB_ERR_ARG;
    if (!ctx->have_fields) return set_err(ctx, LB_ERR_STATE, "no fields");
    int rc = current_forces(ctx);
    if (rc) return rc;
    rc = launched(ctx, launch_totals(ctx->L, ctx->prec, ctx->totals_dev, ctx->stream), "totals kernels");
    if (rc) return rc;
    CK(cudaMemcpyAsync(out, ctx->totals_dev, 64, cudaMemcpyDeviceToHost, ctx->stream), "copy totals");
    CK(cudaStreamSynchronize(ctx->stream), "totals sync");
    return LB_OK;
}

int lb_get_populations(lb_ctx* ctx, int k, double* out) {
    if (!ctx || !out || k < 0 || k >= ctx->L.ncomp) return LB_ERR_ARG;
    if (!ctx->have_fields) return set_err(ctx, LB_ERR_STATE, "no fields");
    Lattice& L = ctx->L;
    // one population plane at a time through the staging area
    double* st = stage_ptr(ctx);
    for (int i = 0; i < Q; i++) {
        int rc = launched(ctx,
                          L.ncomp == 1 ? launch_single_populations_out(L, ctx->prec, i, st, ctx->stream)
                                       : launch_populations_out(L, ctx->prec, k, i, st, ctx->stream),
                          "pops kernel");
        if (rc) return rc;
        CK(cudaMemcpyAsync(out + (size_t)i * L.N, st, (size_t)L.N * 8, cudaMemcpyDeviceToHost, ctx->stream),
           "copy pops");
        CK(cudaStreamSynchronize(ctx->stream), "pops sync");
    }
    return LB_OK;
}

int lb_get_owner(lb_ctx* ctx, int* out) {
    if (!ctx || !out) return LB_ERR_ARG;
    if (ctx->L.ncomp == 1) {  // no particle nodes
        for (long long s = 0; s < ctx->L.N; s++) out[s] = -1;
        return LB_OK;
    }
    CK(cudaMemcpyAsync(out, ctx->L.owner, (size_t)ctx->L.N * 4, cudaMemcpyDeviceToHost, ctx->stream), "copy owner");
    CK(cudaStreamSynchronize(ctx->stream), "owner sync");
    return LB_OK;
}

int lb_get_colloids(lb_ctx* ctx, double* pos, double* vel, double* omega, double* quat, double* force,
                    double* torque) {
    if (!ctx) return LB_ERR_ARG;
    Lattice& L = ctx->L;
    size_t n = (size_t)L.nc;
    cudaStream_t s = ctx->stream;
    if (n) {
        if (pos) CK(cudaMemcpyAsync(pos, L.pos, 24 * n, cudaMemcpyDeviceToHost, s), "copy pos");
        if (vel) CK(cudaMemcpyAsync(vel, L.vel, 24 * n, cudaMemcpyDeviceToHost, s), "copy vel");
        if (omega) CK(cudaMemcpyAsync(omega, L.omg, 24 * n, cudaMemcpyDeviceToHost, s), "copy omega");
        if (quat) CK(cudaMemcpyAsync(quat, L.quat, 32 * n, cudaMemcpyDeviceToHost, s), "copy quat");
        if (force) CK(cudaMemcpyAsync(force, L.Ftot, 24 * n, cudaMemcpyDeviceToHost, s), "copy force");
        if (torque) CK(cudaMemcpyAsync(torque, L.Ttot, 24 * n, cudaMemcpyDeviceToHost, s), "copy torque");
        CK(cudaStreamSynchronize(s), "colloid sync");
    }
    return (int)n;
}

int lb_get_colloid_terms(lb_ctx* ctx, int which, double* out) {
    if (!ctx || !out || which < 0 || which > 10) return LB_ERR_ARG;
    Lattice& L = ctx->L;
    const double* src[11] = {L.Fliq, L.Tliq, L.Fd, L.Td, L.Fc, L.Tc, L.Fs, L.Ts, L.Fpair, L.Ftot, L.Ttot};
    if (L.nc) {
        CK(cudaMemcpyAsync(out, src[which], 24 * (size_t)L.nc, cudaMemcpyDeviceToHost, ctx->stream), "copy term");
        CK(cudaStreamSynchronize(ctx->stream), "term sync");
    }
    return LB_OK;
}

long long lb_launch_count(const lb_ctx* ctx) { return ctx ? ctx->launches : -1; }

long long lb_pair_list_builds(lb_ctx* ctx) {
    if (!ctx) return -1;
    unsigned long long b = 0;
    if (cudaMemcpyAsync(&b, ctx->L.vl_builds, 8, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return -1;
    return (long long)b;
}

int lb_fused_kernel(const lb_ctx* ctx) {
    if (!ctx) return LB_ERR_ARG;
    const bool unit = ctx->L.P.tau[0] == 1.0 && ctx->L.P.tau[1] == 1.0;
    if (ctx->L.ncomp == 1) return LB_FUSED_SINGLE;
    if (unit) return LB_FUSED_MOMENTUM;
    return ctx->L.nc > 0 ? LB_FUSED_TWO_PASS : LB_FUSED_PLAIN;
}


// ------------------------------------------------------------- adjoint

int lb_state_bytes(const lb_ctx* ctx, size_t* bytes) {
    if (!ctx || !bytes) return LB_ERR_ARG;
    *bytes = state_bytes(ctx);
    return LB_OK;
}

int lb_get_state(lb_ctx* ctx, void* d_dst) {
    if (!ctx || !d_dst) return LB_ERR_ARG;
    if (!ctx->have_fields) return set_err(ctx, LB_ERR_STATE, "no fields");
    CK(cudaMemcpyAsync(d_dst, ctx->L.f_cur, state_bytes(ctx), cudaMemcpyDeviceToDevice, ctx->stream), "copy state");
    CK(cudaStreamSynchronize(ctx->stream), "state sync");
    return LB_OK;
}

int lb_set_state(lb_ctx* ctx, const void* d_src) {
    if (!ctx || !d_src) return LB_ERR_ARG;
    if (!ctx->have_fields) return set_err(ctx, LB_ERR_STATE, "no fields");
    CK(cudaMemcpyAsync(ctx->L.f_cur, d_src, state_bytes(ctx), cudaMemcpyDeviceToDevice, ctx->stream), "copy state");
    CK(cudaStreamSynchronize(ctx->stream), "state sync");
    return LB_OK;
}

// scratch: [dJdF: maxc x 3 doubles][gradient accumulator: 8 doubles][seed value: 8 doubles][kernel scratch]
static size_t adj_dJdF_bytes(const lb_ctx* ctx) { return align_up((size_t)(ctx->maxc > 0 ? ctx->maxc : 1) * 24); }
static double* adj_grads(const lb_ctx* ctx, void* scratch) { return (double*)((char*)scratch + adj_dJdF_bytes(ctx)); }
static double* adj_value(const lb_ctx* ctx, void* scratch) {
    return (double*)((char*)scratch + adj_dJdF_bytes(ctx) + align_up(64));
}
static size_t adj_head_bytes(const lb_ctx* ctx) { return adj_dJdF_bytes(ctx) + 2 * align_up(64); }

int lb_adjoint_bytes(const lb_ctx* ctx, size_t* field_bytes, size_t* scratch_bytes) {
    if (!ctx || !field_bytes || !scratch_bytes) return LB_ERR_ARG;
    *field_bytes = adjoint_field_bytes(ctx->L, ctx->prec);
    *scratch_bytes = adj_head_bytes(ctx) + adjoint_scratch_bytes(ctx->L, ctx->prec);
    return LB_OK;
}

static int adjoint_ready(lb_ctx* ctx) {
    if (!ctx->have_fields) return set_err(ctx, LB_ERR_STATE, "no fields");
    if (ctx->L.ncomp == 1) return set_err(ctx, LB_ERR_STATE, "the adjoint is built for the two-component lattice");
    if (ctx->L.sr)
        return set_err(ctx, LB_ERR_STATE, "stochastic rounding: recomputed forward steps would differ from the recorded ones");
    if (!ctx->all_fixed) return set_err(ctx, LB_ERR_STATE, "the adjoint needs immobile particles (infinite mass, at rest)");
    for (int f = 0; f < 2; f++)
        if (ctx->L.P.open[f] == 1 || ctx->L.P.open[f] == 3 || (ctx->L.P.open[f] == 2 && ctx->L.P.open_extrap))
            return set_err(ctx, LB_ERR_STATE, "the adjoint handles walls and velocity faces without extrapolation only");
    return LB_OK;
}

int lb_adjoint_seed(lb_ctx* ctx, double weight, void* d_adj, void* d_scratch, double* value) {
    if (!ctx || !d_adj || !d_scratch || !value) return LB_ERR_ARG;
    int rc = adjoint_ready(ctx);
    if (rc) return rc;
    char* head = (char*)d_scratch;
    double* val_dev = adj_value(ctx, d_scratch);
    // a reverse sweep starts here: clear the gradient accumulator
    CK(cudaMemsetAsync(adj_grads(ctx, d_scratch), 0, 8 * sizeof(double), ctx->stream), "clear gradients");
    rc = launched(ctx, launch_adjoint_seed(ctx->L, ctx->prec, d_adj, head + adj_head_bytes(ctx), weight, val_dev,
                                           ctx->stream), "adjoint seed");
    if (rc) return rc;
    CK(cudaMemcpyAsync(value, val_dev, 8, cudaMemcpyDeviceToHost, ctx->stream), "copy seed value");
    CK(cudaStreamSynchronize(ctx->stream), "seed sync");
    return LB_OK;
}

// the launches of one reverse step; dJdF_dev: device dJ/dF_liq or null
static int adjoint_step_launch(lb_ctx* ctx, const void* d_state, const void* d_adj_in, void* d_adj_out,
                               void* d_scratch, const double* dJdF_dev) {
    Lattice Ls = ctx->L;
    Ls.f_cur = (void*)d_state;
    cudaStream_t s = ctx->stream;
    char* head = (char*)d_scratch;
    // forward densities of step t: rho everywhere, wall and virtual densities
    int n = ensure_link_classes(ctx, s);
    n += launch_density(Ls, ctx->prec, s);
    n += launch_wall_psi(Ls, ctx->prec, s);
    n += launch_virtual(Ls, ctx->prec, 0, s);
    n += launch_adjoint_step(Ls, ctx->prec, d_adj_in, d_adj_out, head + adj_head_bytes(ctx),
                             Ls.nc > 0 ? dJdF_dev : nullptr, adj_grads(ctx, d_scratch), s);
    return launched(ctx, n, "adjoint step");
}

// add the accumulated parameter gradients to grads (host) and clear them
static int adjoint_read_grads(lb_ctx* ctx, void* d_scratch, double* grads) {
    double g[5];
    double* acc = adj_grads(ctx, d_scratch);
    CK(cudaMemcpyAsync(g, acc, 40, cudaMemcpyDeviceToHost, ctx->stream), "copy grads");
    CK(cudaMemsetAsync(acc, 0, 40, ctx->stream), "clear gradients");
    CK(cudaStreamSynchronize(ctx->stream), "adjoint sync");
    for (int a = 0; a < 5; a++) grads[a] += g[a];
    return LB_OK;
}

int lb_adjoint_step(lb_ctx* ctx, const void* d_state, const void* d_adj_in, void* d_adj_out, void* d_scratch,
                    const double* dJdF, double* grads) {
    if (!ctx || !d_state || !d_adj_in || !d_adj_out || !d_scratch || !grads || d_adj_in == d_adj_out)
        return LB_ERR_ARG;
    int rc = adjoint_ready(ctx);
    if (rc) return rc;
    double* dJdF_dev = (double*)d_scratch;
    if (dJdF && ctx->L.nc > 0)
        CK(cudaMemcpyAsync(dJdF_dev, dJdF, (size_t)ctx->L.nc * 24, cudaMemcpyHostToDevice, ctx->stream),
           "copy dJdF");
    rc = adjoint_step_launch(ctx, d_state, d_adj_in, d_adj_out, d_scratch, dJdF ? dJdF_dev : nullptr);
    if (rc) return rc;
    return adjoint_read_grads(ctx, d_scratch, grads);
}

int lb_adjoint_step_async(lb_ctx* ctx, const void* d_state, const void* d_adj_in, void* d_adj_out,
                          void* d_scratch, const double* d_dJdF, double* grads) {
    if (!ctx || !d_state || !d_adj_in || !d_adj_out || !d_scratch || d_adj_in == d_adj_out) return LB_ERR_ARG;
    int rc = adjoint_ready(ctx);
    if (rc) return rc;
    rc = adjoint_step_launch(ctx, d_state, d_adj_in, d_adj_out, d_scratch, d_dJdF);
    if (rc) return rc;
    return grads ? adjoint_read_grads(ctx, d_scratch, grads) : LB_OK;
}

int lb_drag_gradient(lb_ctx* ctx, const double* d_F, double weight, double eps, double* d_dJdF) {
    if (!ctx || !d_F || !d_dJdF || !(eps >= 0.0)) return LB_ERR_ARG;
    return launched(ctx, launch_drag_gradient(ctx->L.nc, d_F, weight, eps, d_dJdF, ctx->stream), "drag gradient");
}

int lb_record(lb_ctx* ctx, void* d_states, double* d_forces, int nsteps) {
    if (!ctx) return LB_ERR_ARG;
    ctx->rec_states = nsteps > 0 ? (char*)d_states : nullptr;
    ctx->rec_forces = nsteps > 0 ? d_forces : nullptr;
    ctx->rec_left = nsteps > 0 ? nsteps : 0;
    ctx->rec_i = 0;
    return LB_OK;
}

int lb_adjoint_initial(lb_ctx* ctx, const void* d_adj, double* d_grad) {
    if (!ctx || !d_adj || !d_grad) return LB_ERR_ARG;
    int rc = adjoint_ready(ctx);
    if (rc) return rc;
    rc = launched(ctx, launch_adjoint_initial(ctx->L, ctx->prec, d_adj, d_grad, ctx->stream), "adjoint initial");
    if (rc) return rc;
    CK(cudaStreamSynchronize(ctx->stream), "initial sync");
    return LB_OK;
}

static int create_events(lb_ctx* ctx, cudaEvent_t** out) {
    cudaEvent_t* ev = new (std::nothrow) cudaEvent_t[2 * PROF_MAX];
    if (!ev) return LB_ERR_NOMEM;
    for (int i = 0; i < 2 * PROF_MAX; i++) {
        cudaError_t e = cudaEventCreate(&ev[i]);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; j++) cudaEventDestroy(ev[j]);
            delete[] ev;
            return cuda_check(ctx, e, "create profile events");
        }
    }
    *out = ev;
    return LB_OK;
}

static void destroy_events(cudaEvent_t*& ev) {
    if (!ev) return;
    for (int i = 0; i < 2 * PROF_MAX; i++) cudaEventDestroy(ev[i]);
    delete[] ev;
    ev = nullptr;
}

int lb_profile(lb_ctx* ctx, int enable) {
    if (!ctx) return LB_ERR_ARG;
    for (int k = 0; enable && k < LB_KERNEL_KINDS; k++)
        if (!ctx->prof_ev[k]) {
            int rc = create_events(ctx, &ctx->prof_ev[k]);
            if (rc) return rc;
        }
    ctx->prof_on = enable ? 1 : 0;
    if (enable)
        for (int k = 0; k < LB_KERNEL_KINDS; k++) ctx->prof_n[k] = 0;
    return LB_OK;
}

int lb_profile_read_kernel(lb_ctx* ctx, int kernel, double* total_ms, long long* launches) {
    if (!ctx || !total_ms || !launches || kernel < 0 || kernel >= LB_KERNEL_KINDS) return LB_ERR_ARG;
    const int n = ctx->prof_n[kernel];
    cudaEvent_t* ev = ctx->prof_ev[kernel];
    double t = 0.0;
    for (int i = 0; i < n; i++) {
        float ms = 0.f;
        CK(cudaEventSynchronize(ev[2 * i + 1]), "profile sync");
        CK(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]), "profile elapsed");
        t += ms;
    }
    *total_ms = t;
    *launches = n;
    return LB_OK;
}

int lb_profile_read(lb_ctx* ctx, double* total_ms, long long* launches) {
    return lb_profile_read_kernel(ctx, LB_KERNEL_FUSED, total_ms, launches);
}

int lb_destroy(lb_ctx* ctx) {
    if (!ctx) return LB_ERR_ARG;
    cudaStreamSynchronize(ctx->stream);
    destroy_side_stream(ctx);
    for (int k = 0; k < LB_KERNEL_KINDS; k++) destroy_events(ctx->prof_ev[k]);
    delete ctx;
    return LB_OK;
}

const char* lb_last_error(const lb_ctx* ctx) { return ctx ? ctx->err : ""; }

}  // extern "C"
