// lbgb_static.cu -- lb_totals_static: the global mass / momentum sums of a
// population array, with its scratch in a file-scope device array instead of
// a caller workspace, so that the call allocates nothing.
//
// Some callers cannot allocate device memory at the point where they want the
// totals: for instance a monitor that runs between the time steps of an
// application whose device memory is managed by its own pool (a raw
// cudaMalloc there would synchronise the device and bypass the pool's
// accounting), and which holds the populations but no library context or
// workspace.  This entry point needs only the caller's populations, node map
// and output buffer.
//
// The scratch is g_plane_partials below: one compensated partial per z-plane.
// It is a __device__ symbol, so its host-side name is only a stand-in: host
// code must not pass it to a kernel.  The first call in each CUDA context
// looks up its device address with cudaGetSymbolAddress and remembers it under
// the context's id (a device reset makes a new context, and the next call a
// new lookup); make that first call before any stream capture.  Every call
// shares the array and leaves the last call's partials in it; each call
// overwrites every partial it reads, so nothing has to start at zero, but two
// calls that overlap on the GPU (different streams, no ordering) race on it.
#include <mutex>

#include "lbgb_internal.cuh"

namespace lbgb {

constexpr int STATIC_MAX_PLANES = 4096;  // nz limit of lb_totals_static
constexpr int STATIC_VALUES = 5;         // mass A, mass B, sum j (3)

// [plane][value][s, c]: 4096 x 5 x 2 doubles = 320 KiB on every device that
// loads the library, held until the process exits
static __device__ __align__(256) double g_plane_partials[STATIC_MAX_PLANES * STATIC_VALUES * 2];

struct StaticArgs {
    const void* pops;
    const uint8_t* mask;
    int nx, ny, nz;
    long long pstride;
    float shift[2];  // FP16 deviation reference rho0^k
};

// one block per z-plane: Neumaier sums of rho^k and j = sum_k sum_i f c
template <int PREC>
__global__ void __launch_bounds__(256) k_static_plane(StaticArgs a, double* partials) {
    typedef typename Prec<PREC>::S S;
    typedef typename Prec<PREC>::C C;
    const S* f = (const S*)a.pops;
    int z = blockIdx.x;
    long long nxy = (long long)a.nx * a.ny, base = nxy * z;
    NSum acc[STATIC_VALUES];
    for (int v = 0; v < STATIC_VALUES; v++) acc[v].s = acc[v].c = 0.0;
    for (long long q = threadIdx.x; q < nxy; q += blockDim.x) {
        long long s = base + q;
        if (a.mask && a.mask[s]) continue;
        for (int k = 0; k < 2; k++) {
            C r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
            for (int i = 0; i < Q; i++) {
                C sh = (sizeof(S) == 2) ? wgt<C>(i) * C(a.shift[k]) : C(0);
                C v = ld_pop(f + ((long long)(k * Q + i)) * a.pstride + s, sh);
                r += v;
                if (cx(i) > 0) jx += v; else if (cx(i) < 0) jx -= v;
                if (cy(i) > 0) jy += v; else if (cy(i) < 0) jy -= v;
                if (cz(i) > 0) jz += v; else if (cz(i) < 0) jz -= v;
            }
            acc[k].add(double(r));
            acc[2].add(double(jx));
            acc[3].add(double(jy));
            acc[4].add(double(jz));
        }
    }
    __shared__ double sh_s[256], sh_c[256];
    for (int v = 0; v < STATIC_VALUES; v++) {
        sh_s[threadIdx.x] = acc[v].s;
        sh_c[threadIdx.x] = acc[v].c;
        __syncthreads();
        if (threadIdx.x == 0) {
            NSum t = {0.0, 0.0};
            for (int q = 0; q < (int)blockDim.x; q++) {
                NSum o = {sh_s[q], sh_c[q]};
                t.merge(o);
            }
            partials[(z * STATIC_VALUES + v) * 2] = t.s;
            partials[(z * STATIC_VALUES + v) * 2 + 1] = t.c;
        }
        __syncthreads();
    }
}

// planes summed in order
__global__ void k_static_final(const double* partials, int nz, double* out) {
    int v = threadIdx.x;
    if (v >= STATIC_VALUES) return;
    NSum t = {0.0, 0.0};
    for (int z = 0; z < nz; z++) {
        NSum o = {partials[(z * STATIC_VALUES + v) * 2], partials[(z * STATIC_VALUES + v) * 2 + 1]};
        t.merge(o);
    }
    out[v] = t.value();
}

// device address of g_plane_partials in the current context, looked up on
// the first call in each context (a context that replaces another on the same
// device, after a device reset, has a new id and gets a fresh lookup)
static double* scratch_address(int device, cudaError_t* err) {
    static std::mutex mu;
    static double* addr[256] = {};
    static unsigned long long ctx[256] = {};
    *err = cudaSuccess;
    if (device < 0 || device >= 256) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device] || !id || ctx[device] != id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_plane_partials);
        if (e != cudaSuccess) {
            *err = e;
            return nullptr;
        }
        addr[device] = (double*)p;
        ctx[device] = id;
    }
    return addr[device];
}

}  // namespace lbgb

extern "C" int lb_totals_static(const void* d_pops, int prec, int nx, int ny, int nz, long long plane_stride,
                                const unsigned char* d_mask, const double* rho0, double* d_out,
                                void* cuda_stream) {
    using namespace lbgb;
    if (!d_pops || !d_out || nx < 1 || ny < 1 || nz < 1) return LB_ERR_ARG;
    if (prec != LB_FP64 && prec != LB_FP32 && prec != LB_FP16) return LB_ERR_ARG;
    if (plane_stride < (long long)nx * ny * nz) return LB_ERR_ARG;
    if (nz > STATIC_MAX_PLANES) return LB_ERR_ARG;  // the static scratch holds 4096 plane partials
    if (prec == LB_FP16 && !rho0) return LB_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LB_ERR_CUDA;
    cudaError_t e;
    double* scratch = scratch_address(dev, &e);
    if (!scratch) return LB_ERR_CUDA;
    StaticArgs a;
    a.pops = d_pops;
    a.mask = (const uint8_t*)d_mask;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.pstride = plane_stride;
    a.shift[0] = rho0 ? float(rho0[0]) : 0.f;
    a.shift[1] = rho0 ? float(rho0[1]) : 0.f;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    switch (prec) {
        case LB_FP64: k_static_plane<LB_FP64><<<nz, 256, 0, st>>>(a, scratch); break;
        case LB_FP32: k_static_plane<LB_FP32><<<nz, 256, 0, st>>>(a, scratch); break;
        default: k_static_plane<LB_FP16><<<nz, 256, 0, st>>>(a, scratch); break;
    }
    k_static_final<<<1, 32, 0, st>>>(scratch, nz, d_out);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}
