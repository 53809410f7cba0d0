// rcx_plan.cu -- host side of librcx.so: plans, scratch, argument checks and the
// launch sequence of the formal solution (C ABI declared in include/rcx.h).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "rcx_internal.h"

namespace {

// Default lane layout of the march: 16 wavelengths per ray, 4 per lane (4 lanes per
// ray, 8 rays of neighbouring directions per warp): the DDA of each lane is shared by
// 4 wavelengths, and a 16-wavelength block of a 1024^2 slab (134 MB of packed field)
// still mostly hits in L2.  Measured fastest of the (block, per-lane) layouts on the
// 1024^2 x 64-wavelength x 8-cascade workload.
constexpr int kDefaultLambdaBlock = 16;
constexpr int kDefaultLambdaPerLane = 4;

thread_local std::string g_last_error;

rc_status fail(rc_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

rc_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return RC_ERR_CUDA;
}

// Makes the plan's device current for the scope and restores the caller's.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(long long v) {
    int s = 0;
    while ((1LL << s) < v) ++s;
    return s;
}

size_t storage_bytes(int precision) { return precision == RC_STORE_F32 ? 4 : 2; }

// Legendre P_n and P_{n-1} at x by the three-term recurrence.
void legendre(int n, double x, double* pn, double* pn1) {
    double p0 = 1.0, p1 = x;
    if (n == 0) {
        *pn = 1.0;
        *pn1 = 0.0;
        return;
    }
    for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *pn1 = p0;
}

// n-point Gauss-Radau rule on [0, 1] in mu = cos(angle to the invariant axis) with the fixed
// node at mu = 0 (the in-plane ray), from the rule on [-1, 1] with fixed node -1: the free
// nodes are the roots of (P_{n-1} + P_n)/(1 + x), found by Newton's method from the
// Chebyshev-Gauss-Radau points; weights 2/n^2 at -1 and (1 - x)/(n P_{n-1}(x))^2.
void gauss_radau(int n, std::vector<double>& mu, std::vector<double>& w) {
    mu.assign(n, 0.0);
    w.assign(n, 0.0);
    if (n == 1) {
        w[0] = 1.0;
        return;
    }
    w[0] = 1.0 / ((double)n * n);                   // (2/n^2) / 2
    for (int k = 1; k < n; ++k) {
        double x = -std::cos(2.0 * M_PI * k / (2.0 * n - 1.0));
        for (int it = 0; it < 100; ++it) {
            double pn, pn1, qn, qn1;
            legendre(n, x, &pn, &pn1);
            const double f = pn + pn1;
            // derivatives: P'_m = m (x P_m - P_{m-1}) / (x^2 - 1)
            legendre(n - 1, x, &qn, &qn1);          // qn = P_{n-1}, qn1 = P_{n-2}
            const double dpn = n * (x * pn - pn1) / (x * x - 1.0);
            const double dpn1 = (n - 1) * (x * qn - qn1) / (x * x - 1.0);
            const double g = f / (1.0 + x);
            const double dg = ((dpn + dpn1) * (1.0 + x) - f) / ((1.0 + x) * (1.0 + x));
            const double dx = g / dg;
            x -= dx;
            if (std::fabs(dx) < 1e-15) break;
        }
        double pn, pn1;
        legendre(n, x, &pn, &pn1);
        mu[k] = 0.5 * (1.0 + x);
        w[k] = 0.5 * (1.0 - x) / ((double)n * n * pn1 * pn1);
    }
}

void free_scratch(rc_plan_s* p) {
    cudaFree(p->d_packed_raw);
    p->d_packed_raw = nullptr;
    p->packed_guard = 0;
    cudaFree(p->d_it);
    p->d_it = nullptr;
    p->it_bytes = 0;
    cudaFree(p->d_R[0]);
    cudaFree(p->d_R[1]);
    cudaFree(p->d_smax);
    cudaFree(p->d_scale);
    p->d_packed = nullptr;
    p->d_R[0] = p->d_R[1] = nullptr;
    p->d_smax = nullptr;
    p->d_scale = nullptr;
    p->packed_bytes = p->R_bytes = 0;
    p->aux_count = 0;
    p->cap_lambda = 0;
}

// Grows the solve scratch to hold n_lambda wavelengths.
// Largest distance from a probe of cascade i to a domain corner (the extreme probes decide).
double far_corner(const rc_plan_s* p, int i) {
    const rcx::LevelGeom& g = p->lv[i];
    const double sp = std::ldexp(1.0, i);
    double far2 = 0.0;
    for (int kx : {0, g.Px - 1})
        for (int kz : {0, g.Pz - 1}) {
            const double x = (kx + 0.5) * sp, z = (kz + 0.5) * sp;
            const double dx = std::max(x, p->nx - x), dz = std::max(z, p->nz - z);
            far2 = std::max(far2, dx * dx + dz * dz);
        }
    return std::sqrt(far2);
}

// Strips of the strip-split march for cascade i (1 = one ordinary launch).  A cascade is
// split when its intervals reach half the domain and one wavelength block of the packed
// field exceeds 96 MiB: such rays cross the whole field within one launch, so with the
// field larger than L2 every voxel is fetched from DRAM many times.  Strips of about 64 MiB
// measured best on the B300 (cascade 5 of 16 wavelengths: 1024^2 10.2 -> 9.7 ms with 2
// strips; 1408^2 42.0 -> 31.3 ms with 4; 1984^2 150 -> 90 ms with 8); shorter cascades lose
// more to the extra launches and the (I, T) traffic than they gain.  rc_options.strips >= 2
// forces a count on every cascade >= 1.
// Cascades >= 1 whose intervals are at most this long (voxels) take the shared-DDA march by
// default: their rays are short, and one DDA walk per 32 rays beats the lane-group march
// (1024^2 x 64 wavelengths: cascade 1, 4 voxels, 1.33 vs 1.56 ms; cascade 2, 16 voxels, 3.05
// vs 3.49 ms).  Longer cascades keep the lane-group march: there the shared DDA's 32 rays in
// flight per warp cost more L2 hits and memory parallelism than its 14-20 % fewer
// instructions save (cascade 3 9.81 vs 9.61 ms, cascade 4 38.9 vs 29.6 ms).
constexpr double kSdMaxInterval = 16.0;

bool use_shared_dda(const rc_plan_s* p, int i, const rcx::LevelArgs& a) {
    if (i == 0 || p->march == RC_MARCH_LANE_GROUP || !rcx::level_sdda_supported(p->LB, p->VL, a))
        return false;
    if (p->march == RC_MARCH_SHARED_DDA_ALL) return true;
    if (p->march == RC_MARCH_TUNED) return (p->march_tuned >> i) & 1u;
    return p->lv[i].b - p->lv[i].a <= kSdMaxInterval;
}

// A wavelength block of the packed field above RCX_SPLIT_MIN_MIB is marched in strips of
// about RCX_STRIP_MIB each on the cascades whose intervals reach half the domain.
#ifndef RCX_SPLIT_MIN_MIB
#define RCX_SPLIT_MIN_MIB 96
#endif
#ifndef RCX_STRIP_MIB
#define RCX_STRIP_MIB 64
#endif
int strips_for_impl(const rc_plan_s* p, int i) {
    if (i == 0 || p->opt.bilinear_fix || p->opt.strips == 1 ||
        !rcx::level_split_supported(p->LB, p->VL))
        return 1;
    if (p->opt.strips >= 2) return std::min(p->opt.strips, p->nx);
    const rcx::LevelGeom& g = p->lv[i];
    const double len = std::min(g.b, far_corner(p, i)) - g.a;   // longest piece in the domain
    if (len < 0.5 * std::max(p->nx, p->nz)) return 1;
    const double block = (double)p->nx * p->nz * p->LB * sizeof(float2);
    constexpr double kSplitMin = RCX_SPLIT_MIN_MIB * double(1 << 20);
    constexpr double kStrip = RCX_STRIP_MIB * double(1 << 20);
    if (block <= kSplitMin) return 1;
    return std::min(std::min(16, p->nx), std::max(2, (int)std::lround(block / kStrip)));
}

// Lambda blocks that one strip launch covers: all of them while their partial (I, T) fits in
// 8 GiB (3 % of the B300's memory).  The hardware hands out CTAs in index order, block after
// block, so the gathers in flight still come from one block's strip; one launch per strip
// instead of one per block and strip leaves one launch tail per strip.  At 2048^2 with 64
// wavelengths (2 GiB of partial state per block) 8 GiB measured 98.2 slices/s against 97.0
// with 2 GiB; 16 GiB gave the same as 8.
#ifndef RCX_IT_BUDGET_GIB
#define RCX_IT_BUDGET_GIB 8
#endif
int split_blocks(size_t per_blk, int n_lblk) {
    constexpr size_t kItBudget = size_t(RCX_IT_BUDGET_GIB) << 30;
    return (int)std::max<size_t>(1, std::min<size_t>((size_t)n_lblk, kItBudget / per_blk));
}

rc_status ensure_scratch(rc_plan_s* p, int n_lambda) {
    n_lambda *= p->n_incl;                           // virtual wavelengths
    if (n_lambda <= p->cap_lambda) return RC_OK;
    const int LB = p->LB;
    const size_t n_lblk = (size_t)((n_lambda + LB - 1) / LB);
    const size_t ncell = (size_t)p->nx * p->nz;
    long long max_rays = 0;
    for (size_t i = 1; i < p->lv.size(); ++i) max_rays = std::max(max_rays, p->lv[i].rays());
    const size_t packed = n_lblk * ncell * LB * sizeof(float2);
    // merged intervals hold one child average per 4 rays
    const size_t Rb = std::max<size_t>(1, n_lblk * (size_t)(max_rays / 4) * LB *
                                              storage_bytes(p->opt.precision));
    // strip-split cascades keep (I, T) per ray and wavelength between launches, for as many
    // lambda blocks as one launch covers (split_blocks)
    size_t itb = 0;
    for (int i = 1; i < p->C; ++i)
        if (strips_for_impl(p, i) > 1) {
            const size_t per_blk = (size_t)p->lv[i].rays() * LB * sizeof(float2);
            itb = std::max(itb, per_blk * split_blocks(per_blk, (int)n_lblk));
        }
    cudaDeviceSynchronize();  // scratch may be in use by work still queued
    free_scratch(p);
    cudaError_t e = cudaSuccess;
    const size_t guard = rcx::packed_guard_bytes(p->nx, LB);
    if ((e = cudaMalloc(&p->d_packed_raw, packed + 2 * guard)) != cudaSuccess ||
        (itb && (e = cudaMalloc(&p->d_it, itb)) != cudaSuccess) ||
        (e = cudaMalloc(&p->d_R[0], Rb)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_R[1], Rb)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_smax, n_lblk * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc(&p->d_scale, n_lblk * sizeof(float))) != cudaSuccess) {
        free_scratch(p);
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? RC_ERR_OOM : RC_ERR_CUDA,
                    std::string("scratch allocation failed: ") + cudaGetErrorString(e));
    }
    p->d_packed = reinterpret_cast<float2*>(reinterpret_cast<char*>(p->d_packed_raw) + guard);
    p->packed_guard = guard;
    p->packed_bytes = packed;
    p->it_bytes = itb;
    p->R_bytes = Rb;
    p->aux_count = n_lblk;
    p->cap_lambda = (int)(n_lblk * LB);
    return RC_OK;
}

// The launch sequence of one solve on device buffers.
// Cascades whose merged intervals are identically zero need no launch: an interval that
// starts beyond the farthest box corner from every probe of its cascade lies entirely in
// free space (I = 0, T = 1, nothing enters: Sec. 3.4), so its R is the merged R of the
// cascade above, and the top cascade's is 0.  Returns the number of cascades from 0 up to
// the highest one that can be non-zero (always >= 1: cascade-0 intervals start at the
// probe).  The bilinear fix retraces to the upper probes, so it keeps every cascade.
int live_cascades(const rc_plan_s* p) {
    if (p->opt.bilinear_fix) return p->C;
    int live = p->C;
    while (live > 1 && p->lv[live - 1].a > far_corner(p, live - 1) * (1.0 + 1e-6) + 1e-3) --live;
    return live;
}

// Rays per CTA of the lane-group march in the plan's current layout.
int lane_group_rays_per_cta(const rc_plan_s* p) {
    return 32 / (p->LB / p->VL) * rcx::kWarpsPerCta;
}

// Lists the CTAs of the highest launched cascade that hold a ray able to reach the box
// (plan creation, synchronous).  The list is kept only when it leaves out at least half
// of the CTAs; otherwise, and on any error, that cascade launches every CTA as before.
void build_top_list(rc_plan_s* p) {
    if (p->opt.bilinear_fix) return;
    const int top = live_cascades(p) - 1;
    if (top < 1) return;
    const rcx::LevelArgs a = rcx::level_args(p, top, 0, nullptr, nullptr, nullptr, nullptr);
    if (!rcx::level_list_supported(p->LB, p->VL, a)) return;
    const int per_cta = lane_group_rays_per_cta(p);
    const long long n_cta = (a.rays + per_cta - 1) / per_cta;
    if (n_cta < 2 || n_cta > 0x7fffffffLL) return;
    // flags, then the count in its own aligned word
    const size_t count_at = ((size_t)n_cta + 15) & ~(size_t)15;
    unsigned char* flags = nullptr;
    int* list = nullptr;
    int hits = -1;
    cudaError_t e = cudaMalloc(&flags, count_at + sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&list, (size_t)n_cta * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(flags, 0, count_at + sizeof(int));
    int* d_count = e == cudaSuccess ? reinterpret_cast<int*>(flags + count_at) : nullptr;
    if (e == cudaSuccess) e = rcx::launch_top_hits(a, per_cta, flags, nullptr);
    if (e == cudaSuccess) e = rcx::launch_compact(flags, n_cta, list, d_count, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(&hits, d_count, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(flags);
    if (e != cudaSuccess || hits < 0 || 2LL * hits > n_cta) {
        cudaFree(list);
        cudaGetLastError();
        return;
    }
    p->d_top_list = list;
    p->top_hits = hits;
    p->top_cascade = top;
    p->top_per_cta = per_cta;
}

rc_status solve_device(rc_plan_s* p, const float* chi, const float* eta, int n_lambda,
                       float* J, float* alo, cudaStream_t s, float* J_eff = nullptr,
                       float* alo_c = nullptr) {
    if (n_lambda == 0) return RC_OK;
    const int n_phys = n_lambda;
    const int NI = p->n_incl;
    if ((long long)n_phys * NI > (1 << 30) || ((long long)n_phys * NI + p->LB - 1) / p->LB > 65535)
        return fail(RC_ERR_ARG, "rc_formal_solve: too many wavelengths for one call (65535 blocks)");
    rc_status st = ensure_scratch(p, n_phys);
    if (st != RC_OK) return st;
    n_lambda = n_phys * NI;                          // virtual wavelengths from here on
    const long long ncell_ = (long long)p->nx * p->nz;
    float* Jv = J;
    float* alov = alo;
    float* Jeffv = J_eff;
    float* alocv = alo_c;
    if (NI > 1) {
        const size_t per = (size_t)n_lambda * ncell_;
        const size_t need = per * (1 + (alo ? 1 : 0) + (J_eff ? 1 : 0) + (alo_c ? 1 : 0));
        if (p->vout_floats < need) {
            cudaDeviceSynchronize();
            cudaFree(p->d_vout);
            p->d_vout = nullptr;
            p->vout_floats = 0;
            if (cudaMalloc(&p->d_vout, need * sizeof(float)) != cudaSuccess) {
                cudaGetLastError();
                return fail(RC_ERR_OOM, "rc_formal_solve: inclination scratch allocation failed");
            }
            p->vout_floats = need;
        }
        float* q = p->d_vout;
        Jv = q;
        q += per;
        if (alo) { alov = q; q += per; }
        if (J_eff) { Jeffv = q; q += per; }
        if (alo_c) { alocv = q; q += per; }
    }
    const int LB = p->LB;
    const int n_lblk = (n_lambda + LB - 1) / LB;
    const long long ncell = (long long)p->nx * p->nz;
    const bool f16 = p->opt.precision != RC_STORE_F32;
    int launches = 0, marks = 0;
    cudaError_t e;
    const bool timing = p->timing && p->ev.size() >= (size_t)(p->C + 7);
    if (timing) {
        p->launch_names.clear();
        cudaEventRecord(p->ev[0], s);
    }
    auto mark = [&](const std::string& name) {   // closes the timed interval of `name`
        if (timing) {
            p->launch_names.push_back(name);
            cudaEventRecord(p->ev[++marks], s);
        }
    };

    if (f16) {
        if ((e = cudaMemsetAsync(p->d_smax, 0, n_lblk * sizeof(unsigned), s)) != cudaSuccess)
            return cuda_fail(e, "memset");
    }
    rcx::PackArgs pa{chi, eta, n_phys, NI, NI > 1 ? p->d_incl : nullptr,
                     p->sparse ? p->d_active : nullptr, ncell, (float)p->voxel, p->d_packed,
                     f16 ? p->d_smax : nullptr};
    if (p->sparse) {
        // cells outside the active set get J = 0 (their lane groups do not run)
        float* outs[4] = {Jv, alov, Jeffv, alocv};
        for (float* o : outs)
            if (o && (e = cudaMemsetAsync(o, 0, (size_t)n_lambda * ncell_ * sizeof(float), s)) != cudaSuccess)
                return cuda_fail(e, "memset");
    }
    if ((e = rcx::launch_pack(LB, n_lblk, pa, s)) != cudaSuccess) return cuda_fail(e, "pack launch");
    ++launches;
    mark("pack");
    if (f16) {
        if ((e = rcx::launch_scales(n_lblk, p->d_smax, p->d_scale, s)) != cudaSuccess)
            return cuda_fail(e, "scale launch");
        ++launches;
        mark("scale");
    }

    const int live = live_cascades(p);
    for (int i = live - 1; i >= 0; --i) {
        rcx::LevelArgs a = rcx::level_args(p, i, n_lambda, Jv, alov, Jeffv, alocv);
        const bool has_up = i < live - 1;
        const int S = strips_for_impl(p, i);
        const bool sdda = use_shared_dda(p, i, a);
        if (S > 1) {
            // one launch per strip, over as many wavelength blocks as it_state holds
            const size_t per_blk = (size_t)a.rays * LB * sizeof(float2);
            const int G = std::max(1, std::min(n_lblk, (int)(p->it_bytes / per_blk)));
            a.it_state = p->d_it;
            a.n_strips = S;
            for (int lb = 0; lb < n_lblk; lb += G)
                for (int ph = 0; ph < S; ++ph) {
                    a.split_lb = lb;
                    a.split_nblk = std::min(G, n_lblk - lb);
                    a.phase = ph;
                    e = sdda ? rcx::launch_level_split_sdda(LB, p->VL, p->opt.precision, has_up, a, s)
                             : rcx::launch_level_split(LB, p->VL, p->opt.precision, has_up, a, s);
                    if (e != cudaSuccess) return cuda_fail(e, "cascade launch (strips)");
                    ++launches;
                }
        } else if (!sdda && !has_up && p->top_list_on && i == p->top_cascade && p->top_hits >= 0 &&
                   !p->sparse &&
                   p->top_per_cta == lane_group_rays_per_cta(p) &&
                   rcx::level_list_supported(LB, p->VL, a)) {
            // the CTAs whose rays all miss the box would store zeros: clear, then march the rest
            const size_t esz = p->opt.precision == RC_STORE_F32 ? 4 : 2;   // FP32, or FP16/BF16
            if ((e = cudaMemsetAsync(a.R_out, 0, (size_t)n_lblk * a.R_out_lstride * esz, s)) != cudaSuccess)
                return cuda_fail(e, "memset");
            e = rcx::launch_level_list(LB, p->VL, p->opt.precision, n_lblk, a, p->d_top_list,
                                       p->top_hits, s);
            if (e != cudaSuccess) return cuda_fail(e, "cascade launch (listed CTAs)");
            if (p->top_hits > 0) ++launches;
        } else {
            e = sdda ? rcx::launch_level_sdda(LB, p->VL, p->opt.precision, has_up, n_lblk, a, s)
                     : rcx::launch_level(LB, p->VL, p->opt.precision, i == 0, has_up, n_lblk, a, s);
            if (e != cudaSuccess) return cuda_fail(e, "cascade launch");
            ++launches;
        }
        mark("cascade " + std::to_string(i));
    }
    if (NI > 1) {
        const float* w = p->d_incl + NI;
        float* outs[4] = {J, alo, J_eff, alo_c};
        const float* ins[4] = {Jv, alov, Jeffv, alocv};
        for (int o = 0; o < 4; ++o) {
            if (!outs[o]) continue;
            if ((e = rcx::launch_incl_reduce(ins[o], outs[o], n_phys, NI, w, ncell_, s)) != cudaSuccess)
                return cuda_fail(e, "inclination reduction launch");
            ++launches;
            mark("inclinations");
        }
    }
    p->last_launches = launches;
    p->timed_launches = timing ? marks : 0;
    return RC_OK;
}

}  // namespace

int rcx::strips_for(const rc_plan_s* p, int i) { return strips_for_impl(p, i); }

int rcx::live_cascade_count(const rc_plan_s* p) { return live_cascades(p); }

rc_status rcx::solve_sequence(rc_plan_s* p, const float* chi, const float* eta, int n_lambda,
                              float* J, cudaStream_t s) {
    if (n_lambda * p->n_incl > p->cap_lambda)
        return fail(RC_ERR_ARG, "solve_sequence: the plan's scratch is too small");
    const bool timing_was = p->timing;
    p->timing = false;
    const rc_status st = solve_device(p, chi, eta, n_lambda, J, nullptr, s);
    p->timing = timing_was;
    return st;
}

rcx::LevelArgs rcx::level_args(const rc_plan_s* p, int i, int n_lambda, float* J, float* alo,
                               float* J_eff, float* alo_c) {
    const rcx::LevelGeom& g = p->lv[i];
    const int LB = p->LB;
    rcx::LevelArgs a{};
    a.field = p->d_packed;
    a.ncell = (long long)p->nx * p->nz;
    a.nx = p->nx;
    a.nz = p->nz;
    a.Px = g.Px;
    a.Pz = g.Pz;
    a.W = (int)g.W;
    a.Wshift = is_pow2(g.W) ? ilog2(g.W) : -1;
    a.spacing = (float)(1 << i);
    a.a = (float)g.a;
    a.b = std::isinf(g.b) ? INFINITY : (float)g.b;
    a.dirs = p->d_dirs + p->dir_off[i];
    // cascade 0 runs one lane group per cell (looping over its directions); sparse plans
    // run the flagged probes only
    if (p->sparse) {
        a.probe_list = p->probe_list[i];
        a.rays = i == 0 ? p->n_flagged[0] : p->n_flagged[i] * g.W;
    } else {
        a.rays = i == 0 ? (long long)p->nx * p->nz : g.rays();
    }
    a.bilinear_fix = p->opt.bilinear_fix;
    if (i < p->C - 1) {
        const rcx::LevelGeom& u = p->lv[i + 1];
        a.a_up = (float)u.a;
        a.R_up = p->d_R[(i + 1) & 1];
        a.Px_up = u.Px;
        a.Pz_up = u.Pz;
        a.R_up_lstride = u.rays() / 4 * LB;       // child averages: one per 4 rays
    }
    if (i > 0) {
        a.R_out = p->d_R[i & 1];
        a.R_out_lstride = g.rays() / 4 * LB;
    }
    a.scale = p->opt.precision != RC_STORE_F32 ? p->d_scale : nullptr;
    a.J = J;
    a.alo = alo;
    a.J_eff = J_eff;
    a.alo_c = alo_c;
    a.n_lambda = n_lambda;
    a.max_steps = p->nx + p->nz + 2;
    return a;
}

rc_status rcx::plan_reserve(rc_plan_s* p, int n_lambda) { return ensure_scratch(p, n_lambda); }

rc_status rcx::plan_set_layout(rc_plan_s* p, int LB, int VL) {
    if (LB == p->LB && VL == p->VL) return RC_OK;
    if (LB != p->LB) {
        const int cap = p->cap_lambda;
        cudaDeviceSynchronize();
        free_scratch(p);
        p->LB = LB;
        p->VL = VL;
        return cap > 0 ? ensure_scratch(p, (cap + p->n_incl - 1) / p->n_incl) : RC_OK;
    }
    p->VL = VL;
    return RC_OK;
}

void rcx::set_last_error(const std::string& msg) { g_last_error = msg; }

extern "C" {

void rc_options_default(rc_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = RC_STORE_F32;
    opt->n_incl = 1;
    opt->interval_rule = 0;
    opt->lambda_block = 0;
    opt->bilinear_fix = 0;
}

const char* rc_last_error(void) { return g_last_error.c_str(); }

const char* rc_status_string(rc_status s) {
    switch (s) {
        case RC_OK: return "RC_OK";
        case RC_ERR_ARG: return "RC_ERR_ARG";
        case RC_ERR_OOM: return "RC_ERR_OOM";
        case RC_ERR_CUDA: return "RC_ERR_CUDA";
        case RC_ERR_TIMEOUT: return "RC_ERR_TIMEOUT";
        case RC_ERR_NOT_CONVERGED: return "RC_ERR_NOT_CONVERGED";
        case RC_ERR_UNSUPPORTED: return "RC_ERR_UNSUPPORTED";
    }
    return "RC_ERR_UNKNOWN";
}

rc_status rc_plan(const rc_grid* grid, int n_cascades, int dirs0, int branching,
                  float interval0, const rc_options* opt, rc_plan_t* out) {
    g_last_error.clear();
    if (!out) return fail(RC_ERR_ARG, "rc_plan: out is NULL");
    *out = nullptr;
    if (!grid) return fail(RC_ERR_ARG, "rc_plan: grid is NULL");
    if (grid->nx < 1 || grid->nz < 1 || grid->nx > (1 << 20) || grid->nz > (1 << 20))
        return fail(RC_ERR_ARG, "rc_plan: nx, nz must be in [1, 2^20]");
    if (!(grid->voxel_size > 0.0) || !std::isfinite(grid->voxel_size))
        return fail(RC_ERR_ARG, "rc_plan: voxel_size must be positive and finite");
    if (n_cascades < 1 || n_cascades > 16) return fail(RC_ERR_ARG, "rc_plan: n_cascades must be in [1, 16]");
    if (dirs0 < 1 || dirs0 > 4096) return fail(RC_ERR_ARG, "rc_plan: dirs0 must be in [1, 4096]");
    if (!(interval0 > 0.0f) || !std::isfinite(interval0))
        return fail(RC_ERR_ARG, "rc_plan: interval0 must be positive and finite");
    if (branching != 4)
        return fail(RC_ERR_UNSUPPORTED, "rc_plan: only branching = 4 (alpha = 2) is implemented");
    rc_options o;
    rc_options_default(&o);
    if (opt) o = *opt;
    if (o.precision < RC_STORE_F32 || o.precision > RC_STORE_BF16)
        return fail(RC_ERR_ARG, "rc_plan: precision must be RC_STORE_F32, _F16 or _BF16");
    if (o.interval_rule != 0 && o.interval_rule != 1)
        return fail(RC_ERR_ARG, "rc_plan: interval_rule must be 0 or 1");
    if (o.n_incl < 1 || o.n_incl > 16) return fail(RC_ERR_ARG, "rc_plan: n_incl must be in [1, 16]");
    if (o.bilinear_fix != 0 && o.bilinear_fix != 1)
        return fail(RC_ERR_ARG, "rc_plan: bilinear_fix must be 0 or 1");
    int LB = o.lambda_block == 0 ? kDefaultLambdaBlock : o.lambda_block;
    if (LB != 1 && LB != 2 && LB != 4 && LB != 8 && LB != 16 && LB != 32)
        return fail(RC_ERR_ARG, "rc_plan: lambda_block must be 0, 1, 2, 4, 8, 16 or 32");
    int VL = o.lambda_per_lane == 0 ? std::min(LB, kDefaultLambdaPerLane) : o.lambda_per_lane;
    if ((VL != 1 && VL != 2 && VL != 4 && VL != 8) || VL > LB)
        return fail(RC_ERR_ARG, "rc_plan: lambda_per_lane must be 0, 1, 2, 4 or 8 and <= lambda_block");
    if (o.strips < 0 || o.strips > 16) return fail(RC_ERR_ARG, "rc_plan: strips must be in [0, 16]");
    if (o.reserved != 0) return fail(RC_ERR_ARG, "rc_plan: reserved option fields must be zero");
    if ((long long)grid->nx * grid->nz * LB >= (1LL << 31))
        return fail(RC_ERR_ARG, "rc_plan: nx * nz * lambda_block must stay below 2^31");

    rc_plan_s* p = new (std::nothrow) rc_plan_s();
    if (!p) return fail(RC_ERR_OOM, "rc_plan: host allocation failed");
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        cudaGetLastError();
        return fail(RC_ERR_CUDA, "rc_plan: no CUDA device");
    }
    p->nx = grid->nx;
    p->nz = grid->nz;
    p->voxel = grid->voxel_size;
    p->C = n_cascades;
    p->W0 = dirs0;
    p->B = branching;
    p->L0 = interval0;
    p->opt = o;
    p->LB = LB;
    p->VL = VL;
    p->n_incl = o.n_incl;

    // geometry (Sec. 2.3, Eq. 12-13), FP64 on the host
    const double g = std::pow(2.0, 0.5 * branching);
    std::vector<float2> dirs;
    double start = 0.0;
    for (int i = 0; i < n_cascades; ++i) {
        rcx::LevelGeom L;
        L.Px = (p->nx + (1 << i) - 1) >> i;
        L.Pz = (p->nz + (1 << i) - 1) >> i;
        L.W = dirs0;
        for (int j = 0; j < i; ++j) L.W *= branching;
        const double len = (double)interval0 * std::pow(g, (double)i);
        if (o.interval_rule == 0) {
            L.a = start;
            L.b = start + len;
            start += len;
        } else {
            L.a = i == 0 ? 0.0 : (double)interval0 * std::pow(g, (double)(i - 1));
            L.b = len;
        }
        if (i == n_cascades - 1) L.b = INFINITY;
        if (L.W > (1LL << 26) || L.rays() > (1LL << 32)) {
            delete p;
            return fail(RC_ERR_ARG, "rc_plan: cascade too large (directions or rays)");
        }
        p->dir_off.push_back(dirs.size());
        for (long long k = 0; k < L.W; ++k) {
            const double th = 2.0 * M_PI * ((double)k + 0.5) / (double)L.W;
            dirs.push_back(make_float2((float)std::cos(th), (float)std::sin(th)));
        }
        p->lv.push_back(L);
    }
    cudaError_t e = cudaMalloc(&p->d_dirs, dirs.size() * sizeof(float2));
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_dirs, dirs.data(), dirs.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && p->n_incl > 1) {
        std::vector<double> mu, w;
        gauss_radau(p->n_incl, mu, w);
        std::vector<float> t(2 * p->n_incl);
        for (int j = 0; j < p->n_incl; ++j) {
            t[j] = (float)(1.0 / std::sqrt(1.0 - mu[j] * mu[j]));
            t[p->n_incl + j] = (float)w[j];
        }
        e = cudaMalloc(&p->d_incl, t.size() * sizeof(float));
        if (e == cudaSuccess)
            e = cudaMemcpy(p->d_incl, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(p->d_dirs);
        delete p;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? fail(RC_ERR_OOM, "rc_plan: direction table allocation failed")
                                              : cuda_fail(e, "rc_plan: direction table upload");
    }
    build_top_list(p);
    *out = p;
    return RC_OK;
}

void rc_plan_destroy(rc_plan_t p) {
    if (!p) return;
    DeviceGuard dg(p->device);
    cudaDeviceSynchronize();
    free_scratch(p);
    cudaFree(p->d_dirs);
    cudaFree(p->d_top_list);
    cudaFree(p->d_incl);
    cudaFree(p->d_vout);
    cudaFree(p->d_active);
    cudaFree(p->d_sparse);
    cudaFree(p->d_stage);
    for (auto& s : p->s_io)
        if (s) cudaStreamDestroy(s);
    for (auto& e : p->io_done)
        if (e) cudaEventDestroy(e);
    for (auto& e : p->ev) cudaEventDestroy(e);
    delete p;
}

rc_status rc_plan_reserve(rc_plan_t p, int n_lambda) {
    g_last_error.clear();
    if (!p) return fail(RC_ERR_ARG, "rc_plan_reserve: plan is NULL");
    if (n_lambda < 0) return fail(RC_ERR_ARG, "rc_plan_reserve: n_lambda < 0");
    DeviceGuard dg(p->device);
    if (!dg.ok) return fail(RC_ERR_CUDA, "rc_plan_reserve: cannot select the plan's device");
    return ensure_scratch(p, n_lambda);
}

size_t rc_plan_scratch_bytes(rc_plan_t p) {
    if (!p) return 0;
    return p->packed_bytes + 2 * p->packed_guard + 2 * p->R_bytes +
           p->aux_count * (sizeof(unsigned) + sizeof(float)) + p->it_bytes + p->stage_bytes;
}

rc_status rc_plan_cascade(rc_plan_t p, int i, int* px, int* pz, long long* dirs, double* a,
                          double* b) {
    if (!p) return fail(RC_ERR_ARG, "rc_plan_cascade: plan is NULL");
    if (i < 0 || i >= p->C) return fail(RC_ERR_ARG, "rc_plan_cascade: cascade index out of range");
    const rcx::LevelGeom& g = p->lv[i];
    if (px) *px = g.Px;
    if (pz) *pz = g.Pz;
    if (dirs) *dirs = g.W;
    if (a) *a = g.a;
    if (b) *b = g.b;
    return RC_OK;
}

int rc_plan_last_launch_count(rc_plan_t p) { return p ? p->last_launches : 0; }

rc_status rc_emergent(rc_plan_t p, const float* chi, const float* eta, int n_lambda,
                      const float* rays, long long n_rays, float mu, float* I, float* contrib,
                      void* stream) {
    g_last_error.clear();
    if (!p) return fail(RC_ERR_ARG, "rc_emergent: plan is NULL");
    if (n_lambda < 0 || n_rays < 0 || !(mu >= 0.0f && mu < 1.0f))
        return fail(RC_ERR_ARG, "rc_emergent: n_lambda, n_rays >= 0 and 0 <= mu < 1 required");
    if (n_lambda == 0 || n_rays == 0) return RC_OK;
    if (!chi || !eta || !rays || !I)
        return fail(RC_ERR_ARG, "rc_emergent: chi, eta, rays and I must be non-NULL");
    if ((reinterpret_cast<uintptr_t>(rays) & 15) != 0)
        return fail(RC_ERR_ARG, "rc_emergent: rays must be 16-byte aligned");
    if ((n_lambda + p->LB - 1) / p->LB > 65535 || n_rays > (1LL << 31))
        return fail(RC_ERR_ARG, "rc_emergent: too many wavelengths or rays");
    DeviceGuard dg(p->device);
    const int NI = p->n_incl;
    rc_status st = ensure_scratch(p, (n_lambda + NI - 1) / NI);   // room for n_lambda packed
    if (st != RC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int LB = p->LB;
    const int n_lblk = (n_lambda + LB - 1) / LB;
    const long long ncell = (long long)p->nx * p->nz;
    // the inclination lengthens the path per projected length by 1/sqrt(1 - mu^2): fold it into
    // the per-voxel opacity and emissivity (S unchanged)
    const double r = 1.0 / std::sqrt(1.0 - (double)mu * mu);
    rcx::PackArgs pa{chi, eta, n_lambda, 1, nullptr, p->sparse ? p->d_active : nullptr, ncell,
                     (float)(p->voxel * r), p->d_packed, nullptr};
    cudaError_t e = rcx::launch_pack(LB, n_lblk, pa, s);
    if (e != cudaSuccess) return cuda_fail(e, "rc_emergent: pack launch");
    rcx::EmergentArgs ea{p->d_packed, ncell, p->nx, p->nz, rays, n_rays, I, contrib, n_lambda,
                         p->nx + p->nz + 2};
    if ((e = rcx::launch_emergent(LB, n_lblk, ea, s)) != cudaSuccess)
        return cuda_fail(e, "rc_emergent: launch");
    p->last_launches = 2;
    return RC_OK;
}

rc_status rc_plan_set_active(rc_plan_t p, const unsigned char* active, void* stream) {
    g_last_error.clear();
    if (!p) return fail(RC_ERR_ARG, "rc_plan_set_active: plan is NULL");
    DeviceGuard dg(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamSynchronize(s);
    cudaFree(p->d_active);
    cudaFree(p->d_sparse);
    p->d_active = nullptr;
    p->d_sparse = nullptr;
    p->sparse = false;
    p->probe_list.clear();
    p->n_flagged.clear();
    if (!active) return RC_OK;
    const int C = p->C;
    const long long ncell = (long long)p->nx * p->nz;
    // layout: [flags of every cascade][lists of every cascade][counts]
    std::vector<size_t> foff(C), loff(C);
    size_t bytes = 0;
    for (int i = 0; i < C; ++i) {
        foff[i] = bytes;
        bytes += ((size_t)p->lv[i].Px * p->lv[i].Pz + 255) & ~(size_t)255;
    }
    for (int i = 0; i < C; ++i) {
        loff[i] = bytes;
        bytes += (((size_t)p->lv[i].Px * p->lv[i].Pz * sizeof(int)) + 255) & ~(size_t)255;
    }
    const size_t coff = bytes;
    bytes += 256;
    cudaError_t e = cudaMalloc(&p->d_sparse, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_active, (size_t)ncell);
    if (e != cudaSuccess) {
        cudaFree(p->d_sparse);
        p->d_sparse = nullptr;
        cudaGetLastError();
        return fail(RC_ERR_OOM, "rc_plan_set_active: allocation failed");
    }
    unsigned char* base = (unsigned char*)p->d_sparse;
    int* counts = (int*)(base + coff);
    e = cudaMemcpyAsync(p->d_active, active, (size_t)ncell, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base, 0, coff, s);
    if (e == cudaSuccess) e = rcx::launch_flags_seed(p->d_active, base + foff[0], ncell, s);
    for (int i = 0; i + 1 < C && e == cudaSuccess; ++i)
        e = rcx::launch_flags_up(base + foff[i], p->lv[i].Px, p->lv[i].Pz, base + foff[i + 1],
                                 p->lv[i + 1].Px, p->lv[i + 1].Pz, s);
    for (int i = 0; i < C && e == cudaSuccess; ++i)
        e = rcx::launch_compact(base + foff[i], (long long)p->lv[i].Px * p->lv[i].Pz,
                                (int*)(base + loff[i]), counts + i, s);
    std::vector<int> h(C);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), counts, C * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "rc_plan_set_active");
    for (int i = 0; i < C; ++i) {
        p->probe_list.push_back((const int*)(base + loff[i]));
        p->n_flagged.push_back(h[i]);
    }
    p->sparse = true;
    return RC_OK;
}

rc_status rc_plan_active_probes(rc_plan_t p, long long* per_cascade) {
    if (!p || !per_cascade) return fail(RC_ERR_ARG, "rc_plan_active_probes: NULL argument");
    for (int i = 0; i < p->C; ++i)
        per_cascade[i] = p->sparse ? p->n_flagged[i] : (long long)p->lv[i].Px * p->lv[i].Pz;
    return RC_OK;
}

rc_status rc_plan_set_lane_layout(rc_plan_t p, int lambda_block, int lambda_per_lane) {
    g_last_error.clear();
    if (!p) return fail(RC_ERR_ARG, "rc_plan_set_lane_layout: plan is NULL");
    const int LB = lambda_block, VL = lambda_per_lane;
    if ((LB != 1 && LB != 2 && LB != 4 && LB != 8 && LB != 16 && LB != 32) ||
        (VL != 1 && VL != 2 && VL != 4 && VL != 8) || VL > LB)
        return fail(RC_ERR_ARG, "rc_plan_set_lane_layout: unsupported layout");
    if ((long long)p->nx * p->nz * LB >= (1LL << 31))
        return fail(RC_ERR_ARG, "rc_plan_set_lane_layout: nx * nz * lambda_block too large");
    DeviceGuard dg(p->device);
    return rcx::plan_set_layout(p, LB, VL);
}

rc_status rc_plan_set_march(rc_plan_t p, int mode) {
    g_last_error.clear();
    if (!p) return fail(RC_ERR_ARG, "rc_plan_set_march: plan is NULL");
    if (mode != RC_MARCH_LANE_GROUP && mode != RC_MARCH_SHARED_DDA &&
        mode != RC_MARCH_SHARED_DDA_ALL)
        return fail(RC_ERR_ARG, "rc_plan_set_march: mode must be RC_MARCH_LANE_GROUP, "
                                "RC_MARCH_SHARED_DDA or RC_MARCH_SHARED_DDA_ALL");
    p->march = mode;
    return RC_OK;
}

rc_status rc_plan_get_march(rc_plan_t p, int* mode) {
    if (!p || !mode) return fail(RC_ERR_ARG, "rc_plan_get_march: NULL argument");
    *mode = p->march;
    return RC_OK;
}

rc_status rc_plan_get_march_cascades(rc_plan_t p, unsigned* mask) {
    if (!p || !mask) return fail(RC_ERR_ARG, "rc_plan_get_march_cascades: NULL argument");
    *mask = 0;
    for (int i = 1; i < p->C && i < 32; ++i) {
        const rcx::LevelArgs a = rcx::level_args(p, i, 1, nullptr, nullptr, nullptr, nullptr);
        if (use_shared_dda(p, i, a)) *mask |= 1u << i;
    }
    return RC_OK;
}

rc_status rc_plan_set_top_list(rc_plan_t p, int enable) {
    if (!p) return fail(RC_ERR_ARG, "rc_plan_set_top_list: plan is NULL");
    if (enable != 0 && enable != 1) return fail(RC_ERR_ARG, "rc_plan_set_top_list: enable must be 0 or 1");
    p->top_list_on = enable != 0;
    return RC_OK;
}

rc_status rc_plan_get_top_list(rc_plan_t p, int* cascade, long long* listed, long long* total) {
    if (!p) return fail(RC_ERR_ARG, "rc_plan_get_top_list: plan is NULL");
    const bool has = p->top_hits >= 0;
    if (cascade) *cascade = has ? p->top_cascade : -1;
    if (listed) *listed = has ? p->top_hits : 0;
    if (total)
        *total = has ? (p->lv[p->top_cascade].rays() + p->top_per_cta - 1) / p->top_per_cta : 0;
    return RC_OK;
}

rc_status rc_plan_get_lane_layout(rc_plan_t p, int* lambda_block, int* lambda_per_lane) {
    if (!p) return fail(RC_ERR_ARG, "rc_plan_get_lane_layout: plan is NULL");
    if (lambda_block) *lambda_block = p->LB;
    if (lambda_per_lane) *lambda_per_lane = p->VL;
    return RC_OK;
}

// Per-cascade choice between the two marches: each is timed per cascade (the tracing events,
// best of two solves after a warm-up) and every cascade keeps the faster.  Leaves the plan in
// RC_MARCH_TUNED when a cascade can take the shared DDA at all.
static rc_status tune_march(rc_plan_t p, const float* chi, const float* eta, int n_lambda,
                            float* J, cudaStream_t s) {
    unsigned can = 0;
    for (int i = 1; i < p->C && i < 32; ++i) {
        const rcx::LevelArgs a = rcx::level_args(p, i, n_lambda, nullptr, nullptr, nullptr, nullptr);
        if (rcx::level_sdda_supported(p->LB, p->VL, a)) can |= 1u << i;
    }
    if (!can) return RC_OK;
    const bool timing_was = p->timing;
    const size_t need = (size_t)p->C + 7;
    while (p->ev.size() < need) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return fail(RC_ERR_CUDA, "rc_plan_autotune: event creation");
        }
        p->ev.push_back(e);
    }
    std::vector<float> best[2];
    const int modes[2] = {RC_MARCH_LANE_GROUP, RC_MARCH_SHARED_DDA_ALL};
    const int mode_was = p->march;
    rc_status st = RC_OK;
    for (int m = 0; m < 2 && st == RC_OK; ++m) {
        p->march = modes[m];
        best[m].assign(p->C, INFINITY);
        p->timing = false;
        st = solve_device(p, chi, eta, n_lambda, J, nullptr, s);      // warm-up
        for (int r = 0; r < 2 && st == RC_OK; ++r) {
            p->timing = true;
            st = solve_device(p, chi, eta, n_lambda, J, nullptr, s);
            if (st != RC_OK) break;
            if (cudaEventSynchronize(p->ev[p->timed_launches]) != cudaSuccess) {
                cudaGetLastError();
                st = fail(RC_ERR_CUDA, "rc_plan_autotune: timing");
                break;
            }
            for (int j = 0; j < p->timed_launches; ++j) {
                const std::string& nm = p->launch_names[j];
                if (nm.rfind("cascade ", 0) != 0) continue;
                const int i = std::atoi(nm.c_str() + 8);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, p->ev[j], p->ev[j + 1]);
                if (i >= 0 && i < p->C) best[m][i] = std::min(best[m][i], ms);
            }
        }
    }
    p->timing = timing_was;
    if (st != RC_OK) {
        p->march = mode_was;
        return st;
    }
    p->march_tuned = 0;
    for (int i = 1; i < p->C && i < 32; ++i)
        if (((can >> i) & 1u) && best[1][i] < best[0][i]) p->march_tuned |= 1u << i;
    p->march = RC_MARCH_TUNED;
    return RC_OK;
}

rc_status rc_plan_autotune(rc_plan_t p, const float* chi, const float* eta, int n_lambda,
                           float* J, void* stream, int* lambda_block, int* lambda_per_lane) {
    g_last_error.clear();
    if (!p || !chi || !eta || !J || n_lambda < 1)
        return fail(RC_ERR_ARG, "rc_plan_autotune: NULL argument or n_lambda < 1");
    DeviceGuard dg(p->device);
    static const int cand[][2] = {{16, 4}, {8, 4}, {32, 4}, {8, 2}, {4, 4}, {4, 2}, {4, 1},
                                  {2, 2}, {1, 1}};
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool timing_was = p->timing;
    p->timing = false;
    float best = INFINITY;
    int bLB = p->LB, bVL = p->VL;
    for (const auto& c : cand) {
        // blocks much wider than the wavelength count only pad with empty lanes
        if (c[0] > 4 && c[0] > 2 * n_lambda) continue;
        if ((long long)p->nx * p->nz * c[0] >= (1LL << 31)) continue;
        rc_status st = rcx::plan_set_layout(p, c[0], c[1]);
        if (st == RC_OK) st = ensure_scratch(p, n_lambda);
        if (st == RC_OK) st = solve_device(p, chi, eta, n_lambda, J, nullptr, s);  // warm-up
        if (st != RC_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            p->timing = timing_was;
            return st;
        }
        cudaEventRecord(e0, s);
        for (int r = 0; r < 2; ++r) solve_device(p, chi, eta, n_lambda, J, nullptr, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            bLB = c[0];
            bVL = c[1];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->timing = timing_was;
    rc_status st = rcx::plan_set_layout(p, bLB, bVL);
    if (st == RC_OK) st = ensure_scratch(p, n_lambda);
    if (st == RC_OK && p->march != RC_MARCH_LANE_GROUP) st = tune_march(p, chi, eta, n_lambda, J, s);
    if (lambda_block) *lambda_block = bLB;
    if (lambda_per_lane) *lambda_per_lane = bVL;
    cudaError_t err = cudaGetLastError();
    if (st == RC_OK && err != cudaSuccess) return cuda_fail(err, "rc_plan_autotune");
    return st;
}

rc_status rc_plan_set_timing(rc_plan_t p, int enable) {
    g_last_error.clear();
    if (!p) return fail(RC_ERR_ARG, "rc_plan_set_timing: plan is NULL");
    DeviceGuard dg(p->device);
    const size_t need = (size_t)p->C + 7;  // pack, scale, C cascades, 4 reductions, start
    while (enable && p->ev.size() < need) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return cuda_fail(err, "rc_plan_set_timing");
        p->ev.push_back(e);
    }
    p->timing = enable != 0;
    p->timed_launches = 0;
    return RC_OK;
}

rc_status rc_plan_launch_times(rc_plan_t p, float* ms, int max_n, int* n_out) {
    g_last_error.clear();
    if (!p || !ms || !n_out) return fail(RC_ERR_ARG, "rc_plan_launch_times: NULL argument");
    if (!p->timing || p->timed_launches == 0)
        return fail(RC_ERR_ARG, "rc_plan_launch_times: no timed solve (enable timing first)");
    DeviceGuard dg(p->device);
    cudaError_t e = cudaEventSynchronize(p->ev[p->timed_launches]);
    if (e != cudaSuccess) return cuda_fail(e, "rc_plan_launch_times");
    const int n = std::min(max_n, p->timed_launches);
    for (int j = 0; j < n; ++j) {
        e = cudaEventElapsedTime(&ms[j], p->ev[j], p->ev[j + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "rc_plan_launch_times");
    }
    *n_out = n;
    return RC_OK;
}

const char* rc_plan_launch_name(rc_plan_t p, int i) {
    if (!p || i < 0 || i >= (int)p->launch_names.size()) return "";
    return p->launch_names[i].c_str();
}

rc_status rc_formal_solve(rc_plan_t p, const float* chi, const float* eta, int n_lambda, float* J,
                          float* alo, void* stream) {
    g_last_error.clear();
    if (!p) return fail(RC_ERR_ARG, "rc_formal_solve: plan is NULL");
    if (alo && p->opt.bilinear_fix)
        return fail(RC_ERR_UNSUPPORTED, "rc_formal_solve: the diagonal operator is defined for "
                                        "the basic construction, not with the bilinear fix");
    if (n_lambda < 0) return fail(RC_ERR_ARG, "rc_formal_solve: n_lambda < 0");
    if (n_lambda > 0 && (!chi || !eta || !J))
        return fail(RC_ERR_ARG, "rc_formal_solve: chi, eta and J must be non-NULL");
    DeviceGuard dg(p->device);
    if (!dg.ok) return fail(RC_ERR_CUDA, "rc_formal_solve: cannot select the plan's device");
    cudaError_t sticky = cudaGetLastError();
    if (sticky != cudaSuccess) return cuda_fail(sticky, "rc_formal_solve: pending CUDA error");
    return solve_device(p, chi, eta, n_lambda, J, alo, (cudaStream_t)stream);
}

rc_status rc_formal_solve_mali(rc_plan_t p, const float* chi, const float* eta, int n_lambda,
                               float* J, float* alo, float* J_eff, float* alo_c, void* stream) {
    g_last_error.clear();
    if (!p) return fail(RC_ERR_ARG, "rc_formal_solve_mali: plan is NULL");
    if (p->opt.bilinear_fix)
        return fail(RC_ERR_UNSUPPORTED, "rc_formal_solve_mali: the MALI outputs are defined "
                                        "for the basic construction, not with the bilinear fix");
    if (n_lambda < 0) return fail(RC_ERR_ARG, "rc_formal_solve_mali: n_lambda < 0");
    if (n_lambda > 0 && (!chi || !eta || !J))
        return fail(RC_ERR_ARG, "rc_formal_solve_mali: chi, eta and J must be non-NULL");
    if (J_eff || alo_c) {
        // the first piece of every cascade-0 ray must be the whole centre-to-edge segment
        double dmax = 0.0;
        for (int k = 0; k < p->W0; ++k) {
            const double th = 2.0 * M_PI * ((double)k + 0.5) / (double)p->W0;
            dmax = std::max(dmax, 0.5 / std::max(std::fabs(std::cos(th)), std::fabs(std::sin(th))));
        }
        if (p->lv[0].b < dmax)
            return fail(RC_ERR_ARG, "rc_formal_solve_mali: the cascade-0 interval is shorter than "
                                    "the centre-to-edge path of a cell");
    }
    DeviceGuard dg(p->device);
    if (!dg.ok) return fail(RC_ERR_CUDA, "rc_formal_solve_mali: cannot select the plan's device");
    cudaError_t sticky = cudaGetLastError();
    if (sticky != cudaSuccess) return cuda_fail(sticky, "rc_formal_solve_mali: pending CUDA error");
    return solve_device(p, chi, eta, n_lambda, J, alo, (cudaStream_t)stream, J_eff, alo_c);
}

// Enqueues a host-buffer solve on the plan's three streams without waiting for it.
static rc_status enqueue_host_solve(rc_plan_t p, const float* chi_h, const float* eta_h,
                                    int n_lambda, float* J_h, float* alo_h, bool pipelined,
                                    const char* who) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, (std::string(who) + ": pending CUDA error").c_str());

    // Chunks of whole lambda blocks; chunk c's copies overlap chunk c-1's solve.  In a
    // blocking call the first chunk (whose copy in nothing hides) and the last (whose copy
    // out nothing hides) are the small unit of about 16 wavelengths; the ones between are
    // twice that, so fewer solves (fewer launch tails) cover the middle.  Pipelined calls
    // hide those copies behind the neighbouring calls' solves instead, so they take chunks of
    // up to four units (one solve per 64 wavelengths).
    const size_t ncell = (size_t)p->nx * p->nz;
    const int LB = p->LB;
    const int unit = std::max(LB, ((16 + LB - 1) / LB) * LB);
    std::vector<int> bounds{0};                                // chunk c: [bounds[c], bounds[c+1])
    while (bounds.back() < n_lambda) {
        const int l0 = bounds.back(), left = n_lambda - l0;
        if (pipelined) {
            bounds.push_back(l0 + std::min(4 * unit, left));
            continue;
        }
        // middle chunks: whole blocks, leaving at least one unit for the last chunk
        const int mid = std::min(2 * unit, (left - unit) / LB * LB);
        bounds.push_back(l0 + ((l0 == 0 || mid <= unit) ? std::min(unit, left) : mid));
    }
    const int n_chunks = (int)bounds.size() - 1;
    int chunk = 0;
    for (int c = 0; c < n_chunks; ++c) chunk = std::max(chunk, bounds[c + 1] - bounds[c]);
    const size_t slab = (size_t)chunk * ncell;                 // floats per array per chunk
    const size_t per_buf = slab * (alo_h ? 4 : 3);             // chi, eta, J (, alo)
    const size_t need = 2 * per_buf * sizeof(float);
    if (p->stage_bytes < need) {
        cudaDeviceSynchronize();                               // earlier solves may use it
        cudaFree(p->d_stage);
        p->d_stage = nullptr;
        p->stage_bytes = 0;
        if ((e = cudaMalloc(&p->d_stage, need)) != cudaSuccess) {
            cudaGetLastError();
            return fail(RC_ERR_OOM, (std::string(who) + ": staging allocation failed").c_str());
        }
        p->stage_bytes = need;
    }
    for (auto& s : p->s_io)
        if (!s && (e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, (std::string(who) + ": stream creation").c_str());
    for (auto& ev : p->io_done)
        if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, (std::string(who) + ": event creation").c_str());
    rc_status st = ensure_scratch(p, chunk);
    if (st != RC_OK) return st;

    // s_io[0] carries copies in, s_io[1] the solves, s_io[2] copies out, so the copy of
    // chunk c's J overlaps chunk c+1's solve.  Chunks are counted across calls: buffer
    // b = count % 2 is reused two chunks later, after its J has left (io_done[b]), so the
    // first chunk of a call copies in while the previous call's last chunk is solved.
    cudaEvent_t loaded[2], solved[2];
    for (int b = 0; b < 2; ++b) {
        cudaEventCreateWithFlags(&loaded[b], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&solved[b], cudaEventDisableTiming);
    }
    int launches = 0;
    const bool timing_was = p->timing;
    p->timing = false;
    for (int c = 0; c < n_chunks && st == RC_OK; ++c) {
        const long long g = p->io_chunks++;
        const int b = (int)(g & 1);
        const int l0 = bounds[c];
        const int nl = bounds[c + 1] - l0;
        const size_t bytes = (size_t)nl * ncell * sizeof(float);
        float* dchi = p->d_stage + b * per_buf;
        float* deta = dchi + slab;
        float* dJ = deta + slab;
        float* dalo = alo_h ? dJ + slab : nullptr;
        if (g >= 2) cudaStreamWaitEvent(p->s_io[0], p->io_done[b], 0);
        cudaMemcpyAsync(dchi, chi_h + (size_t)l0 * ncell, bytes, cudaMemcpyHostToDevice, p->s_io[0]);
        cudaMemcpyAsync(deta, eta_h + (size_t)l0 * ncell, bytes, cudaMemcpyHostToDevice, p->s_io[0]);
        cudaEventRecord(loaded[b], p->s_io[0]);
        cudaStreamWaitEvent(p->s_io[1], loaded[b], 0);
        st = solve_device(p, dchi, deta, nl, dJ, dalo, p->s_io[1]);
        launches += p->last_launches;
        cudaEventRecord(solved[b], p->s_io[1]);
        cudaStreamWaitEvent(p->s_io[2], solved[b], 0);
        cudaMemcpyAsync(J_h + (size_t)l0 * ncell, dJ, bytes, cudaMemcpyDeviceToHost, p->s_io[2]);
        if (alo_h)
            cudaMemcpyAsync(alo_h + (size_t)l0 * ncell, dalo, bytes, cudaMemcpyDeviceToHost, p->s_io[2]);
        cudaEventRecord(p->io_done[b], p->s_io[2]);
    }
    // events recorded on a stream may be destroyed at once (released when they complete)
    for (int b = 0; b < 2; ++b) {
        cudaEventDestroy(loaded[b]);
        cudaEventDestroy(solved[b]);
    }
    p->last_launches = launches;
    p->timing = timing_was;
    if (st != RC_OK) return st;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, who);
    return RC_OK;
}

static rc_status wait_host_solves(rc_plan_t p, const char* who) {
    cudaError_t e = cudaSuccess;
    for (int k = 2; k >= 0; --k)
        if (p->s_io[k]) {
            const cudaError_t ek = cudaStreamSynchronize(p->s_io[k]);
            if (e == cudaSuccess) e = ek;
        }
    return e == cudaSuccess ? RC_OK : cuda_fail(e, who);
}

static rc_status check_host_args(rc_plan_t p, const float* chi_h, const float* eta_h,
                                 int n_lambda, const float* J_h, const char* who) {
    if (!p) return fail(RC_ERR_ARG, (std::string(who) + ": plan is NULL").c_str());
    if (n_lambda < 0) return fail(RC_ERR_ARG, (std::string(who) + ": n_lambda < 0").c_str());
    if (n_lambda > 0 && (!chi_h || !eta_h || !J_h))
        return fail(RC_ERR_ARG, (std::string(who) + ": chi, eta and J must be non-NULL").c_str());
    return RC_OK;
}

rc_status rc_formal_solve_host(rc_plan_t p, const float* chi_h, const float* eta_h, int n_lambda,
                               float* J_h, float* alo_h) {
    g_last_error.clear();
    rc_status st = check_host_args(p, chi_h, eta_h, n_lambda, J_h, "rc_formal_solve_host");
    if (st != RC_OK || n_lambda == 0) return st;
    DeviceGuard dg(p->device);
    if (!dg.ok) return fail(RC_ERR_CUDA, "rc_formal_solve_host: cannot select the plan's device");
    st = enqueue_host_solve(p, chi_h, eta_h, n_lambda, J_h, alo_h, false, "rc_formal_solve_host");
    const rc_status sw = wait_host_solves(p, "rc_formal_solve_host");
    return st != RC_OK ? st : sw;
}

rc_status rc_formal_solve_host_async(rc_plan_t p, const float* chi_h, const float* eta_h,
                                     int n_lambda, float* J_h, float* alo_h) {
    g_last_error.clear();
    rc_status st = check_host_args(p, chi_h, eta_h, n_lambda, J_h, "rc_formal_solve_host_async");
    if (st != RC_OK || n_lambda == 0) return st;
    DeviceGuard dg(p->device);
    if (!dg.ok) return fail(RC_ERR_CUDA, "rc_formal_solve_host_async: cannot select the plan's device");
    return enqueue_host_solve(p, chi_h, eta_h, n_lambda, J_h, alo_h, true,
                              "rc_formal_solve_host_async");
}

rc_status rc_plan_wait(rc_plan_t p) {
    g_last_error.clear();
    if (!p) return fail(RC_ERR_ARG, "rc_plan_wait: plan is NULL");
    DeviceGuard dg(p->device);
    if (!dg.ok) return fail(RC_ERR_CUDA, "rc_plan_wait: cannot select the plan's device");
    return wait_host_solves(p, "rc_plan_wait");
}

}  // extern "C"
