// rcx_noalloc.cu -- rc_formal_solve_noalloc: the formal solution for callers that
// cannot allocate device memory.
//
// Its scratch (direction tables, packed field, two cascades of merged intervals)
// lives in one file-scope __device__ array of kNoallocScratchBytes, which every
// GPU that loads librcx.so holds until the process exits.  Host code never uses
// the array's name as an address: the first call on a device (with that device
// current) asks the runtime for the array's device address with
// cudaGetSymbolAddress, checks the result and caches it for that device together
// with the unique ID of the CUDA context it belongs to.  A later call that finds
// another context current (after cudaDeviceReset, or after the primary context was
// released and created again, which reloads the module and can move the array)
// looks the address up again instead of launching on a stale pointer.
#include <cuda.h>   // CUcontext / CUresult types only; the entry points are fetched at run time

#include <cmath>
#include <mutex>
#include <string>

#include "rcx_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)32 << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};   // context ID the address belongs to

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

rc_status nfail(rc_status s, const std::string& m) {
    rcx::set_last_error(m);
    return s;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Direction tables of every cascade: theta = 2 pi (k + 1/2) / W, written in place.
__global__ void noalloc_dirs_kernel(float2* dirs, long long W, long long off) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= W) return;
    double s, c;
    sincospi((2.0 * (double)k + 1.0) / (double)W, &s, &c);
    dirs[off + k] = make_float2((float)c, (float)s);
}

// Unique ID of the current CUDA context (IDs are never reused within a process), or 0
// when the driver cannot give one; called with g_setup_mutex held.
unsigned long long current_context_id() {
    static bool looked_up = false;
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!looked_up) {
        looked_up = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array on the current device.  Looked up once per device
// and context; with no context ID to compare (an old driver), looked up on every call.
rc_status scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return nfail(RC_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lk(g_setup_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            g_scratch_addr[dev] = nullptr;
            return nfail(RC_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array: ") +
                                          cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return RC_OK;
}

}  // namespace

extern "C" rc_status rc_formal_solve_noalloc(const rc_grid* grid, int n_cascades, int dirs0,
                                             float interval0, const float* chi, const float* eta,
                                             int n_lambda, float* J, float* alo, void* stream) {
    rcx::set_last_error("");
    if (!grid) return nfail(RC_ERR_ARG, "rc_formal_solve_noalloc: grid is NULL");
    const int nx = grid->nx, nz = grid->nz;
    if (nx < 1 || nz < 1 || nx > (1 << 20) || nz > (1 << 20))
        return nfail(RC_ERR_ARG, "rc_formal_solve_noalloc: nx, nz must be in [1, 2^20]");
    if (!(grid->voxel_size > 0.0) || !std::isfinite(grid->voxel_size))
        return nfail(RC_ERR_ARG, "rc_formal_solve_noalloc: voxel_size must be positive and finite");
    if (n_cascades < 1 || n_cascades > 16)
        return nfail(RC_ERR_ARG, "rc_formal_solve_noalloc: n_cascades must be in [1, 16]");
    if (dirs0 < 1 || dirs0 > 4096)
        return nfail(RC_ERR_ARG, "rc_formal_solve_noalloc: dirs0 must be in [1, 4096]");
    if (!(interval0 > 0.0f) || !std::isfinite(interval0))
        return nfail(RC_ERR_ARG, "rc_formal_solve_noalloc: interval0 must be positive and finite");
    if (n_lambda < 0) return nfail(RC_ERR_ARG, "rc_formal_solve_noalloc: n_lambda < 0");
    if (n_lambda == 0) return RC_OK;
    if (!chi || !eta || !J)
        return nfail(RC_ERR_ARG, "rc_formal_solve_noalloc: chi, eta and J must be non-NULL");

    // geometry of the cascades (rule 0 intervals, branching 4), and the scratch it needs
    constexpr int LB = 4, VL = 2;
    const int n_lblk = (n_lambda + LB - 1) / LB;
    if (n_lblk > 65535) return nfail(RC_ERR_ARG, "rc_formal_solve_noalloc: too many wavelengths");
    const long long ncell = (long long)nx * nz;
    rcx::LevelGeom lv[16];
    long long dir_off[16];
    long long n_dirs = 0, max_rays = 0;
    double start = 0.0;
    for (int i = 0; i < n_cascades; ++i) {
        lv[i].Px = (nx + (1 << i) - 1) >> i;
        lv[i].Pz = (nz + (1 << i) - 1) >> i;
        lv[i].W = dirs0;
        for (int j = 0; j < i; ++j) lv[i].W *= 4;
        if (lv[i].W > (1LL << 26))
            return nfail(RC_ERR_ARG, "rc_formal_solve_noalloc: too many directions");
        const double len = (double)interval0 * std::pow(4.0, (double)i);
        lv[i].a = start;
        lv[i].b = i == n_cascades - 1 ? INFINITY : start + len;
        start += len;
        dir_off[i] = n_dirs;
        n_dirs += lv[i].W;
        if (i > 0) max_rays = std::max(max_rays, lv[i].rays());
    }
    const size_t dirs_bytes = align256((size_t)n_dirs * sizeof(float2));
    const size_t packed_bytes = align256((size_t)n_lblk * ncell * LB * sizeof(float2));
    const size_t guard = rcx::packed_guard_bytes(nx, LB);   // around the field (march prefetch)
    const size_t R_bytes = align256((size_t)n_lblk * (size_t)(max_rays / 4) * LB * sizeof(float));
    const size_t need = dirs_bytes + guard + packed_bytes + guard + 2 * R_bytes;
    if (need > kNoallocScratchBytes)
        return nfail(RC_ERR_ARG, "rc_formal_solve_noalloc: this problem needs " +
                                     std::to_string(need) + " bytes of scratch, more than the " +
                                     std::to_string(kNoallocScratchBytes) +
                                     "-byte static array; use rc_plan + rc_formal_solve");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nfail(RC_ERR_CUDA, "rc_formal_solve_noalloc: no current CUDA device");
    }
    unsigned char* base = nullptr;
    rc_status st = scratch_address(dev, &base);
    if (st != RC_OK) return st;
    float2* dirs = reinterpret_cast<float2*>(base);
    float2* packed = reinterpret_cast<float2*>(base + dirs_bytes + guard);
    unsigned char* after = base + dirs_bytes + guard + packed_bytes + guard;
    float* R[2] = {reinterpret_cast<float*>(after), reinterpret_cast<float*>(after + R_bytes)};
    cudaStream_t s = (cudaStream_t)stream;

    // Everything below overwrites what it later reads; nothing has to start at zero.
    for (int i = 0; i < n_cascades; ++i) {
        noalloc_dirs_kernel<<<(unsigned)((lv[i].W + 255) / 256), 256, 0, s>>>(dirs, lv[i].W, dir_off[i]);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return nfail(RC_ERR_CUDA, std::string("rc_formal_solve_noalloc: ") + cudaGetErrorString(e));
    }
    rcx::PackArgs pa{chi, eta, n_lambda, 1, nullptr, nullptr, ncell, (float)grid->voxel_size,
                     packed, nullptr};
    if ((e = rcx::launch_pack(LB, n_lblk, pa, s)) != cudaSuccess)
        return nfail(RC_ERR_CUDA, std::string("rc_formal_solve_noalloc: ") + cudaGetErrorString(e));
    for (int i = n_cascades - 1; i >= 0; --i) {
        rcx::LevelArgs a{};
        a.field = packed;
        a.ncell = ncell;
        a.nx = nx;
        a.nz = nz;
        a.Px = lv[i].Px;
        a.Pz = lv[i].Pz;
        a.W = (int)lv[i].W;
        a.Wshift = -1;
        if ((lv[i].W & (lv[i].W - 1)) == 0) {
            a.Wshift = 0;
            while ((1LL << a.Wshift) < lv[i].W) ++a.Wshift;
        }
        a.spacing = (float)(1 << i);
        a.a = (float)lv[i].a;
        a.b = std::isinf(lv[i].b) ? INFINITY : (float)lv[i].b;
        a.dirs = dirs + dir_off[i];
        a.rays = i == 0 ? ncell : lv[i].rays();   // cascade 0 runs one lane group per cell
        const bool has_up = i < n_cascades - 1;
        if (has_up) {
            a.R_up = R[(i + 1) & 1];
            a.Px_up = lv[i + 1].Px;
            a.Pz_up = lv[i + 1].Pz;
            a.R_up_lstride = lv[i + 1].rays() / 4 * LB;   // child averages
        }
        if (i > 0) {
            a.R_out = R[i & 1];
            a.R_out_lstride = lv[i].rays() / 4 * LB;
        }
        a.J = J;
        a.alo = alo;
        a.n_lambda = n_lambda;
        a.max_steps = nx + nz + 2;
        if ((e = rcx::launch_level(LB, VL, RC_STORE_F32, i == 0, has_up, n_lblk, a, s)) != cudaSuccess)
            return nfail(RC_ERR_CUDA, std::string("rc_formal_solve_noalloc: ") + cudaGetErrorString(e));
    }
    return RC_OK;
}
