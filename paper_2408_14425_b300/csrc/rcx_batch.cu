// rcx_batch.cu -- many independent formal solutions (domains of uneven sizes, each with
// its own wavelength count) captured once in a CUDA graph.  A domain that fills the GPU on
// its own (at least kSoloWaves waves of CTAs in every live cascade) runs its own launch
// sequence, as rc_formal_solve would: its cascades follow one another while the merged
// intervals they pass on are still in L2, and its free-space cascades are skipped.  The
// smaller domains share one launch per cascade over a work list of CTA-sized chunks,
// segments sorted by estimated cost.  An optional native autotuner picks the lane layout by
// timing graph replays of the candidates on a sample of the batch (the first wavelength
// block of each domain).
#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "rcx_internal.h"

namespace {

rc_status bfail(rc_status s, const std::string& m) {
    rcx::set_last_error(m);
    return s;
}
rc_status bcuda(cudaError_t e, const char* what) {
    cudaGetLastError();
    rcx::set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    return RC_ERR_CUDA;
}

struct LevelTables {
    std::vector<long long> prefix;
    std::vector<int> dom, lblk;
    long long total = 0;
};

}  // namespace

struct rc_batch_s {
    int device = 0;
    int n = 0, C = 0;
    std::vector<rc_plan_t> plans;
    std::vector<const float*> chi, eta;
    std::vector<float*> J;
    std::vector<int> nl;
    // device tables: [C] level arg arrays, pack args, segment tables
    void* d_tables = nullptr;
    std::vector<rcx::BatchLevelArgs> level;    // index i = cascade
    rcx::BatchPackArgs pack{};
    std::vector<int> grid;                     // per cascade
    int pack_grid = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<char> solo;                    // per domain: runs its own launch sequence
    int launches = 0;
    int LB = 0, VL = 0, precision = 0;
};

namespace {

void release(rc_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    cudaFree(b->d_tables);
    b->d_tables = nullptr;
}

// Builds the device tables for the plans' current lane layout and captures the graph.
// With first_block_only the tables hold only the first lambda block of every domain (the
// autotuner's sample of the workload).
rc_status build(rc_batch_s* b, bool first_block_only = false) {
    release(b);
    const int n = b->n, C = b->C;
    rc_plan_s* p0 = b->plans[0];
    b->LB = p0->LB;
    b->VL = p0->VL;
    b->precision = p0->opt.precision;
    const int LB = b->LB;
    for (int d = 0; d < n; ++d) {
        rc_status st = rcx::plan_reserve(b->plans[d], b->nl[d]);
        if (st != RC_OK) return st;
    }
    // domains that fill the GPU alone: every live cascade has kSoloWaves waves of CTAs (the
    // march kernels keep up to 48 warps on an SM)
    constexpr int kSoloWaves = 4, kCtasPerSm = 48 / rcx::kWarpsPerCta;
    const int G_rays = 32 / (LB / b->VL) * rcx::kWarpsPerCta;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    const long long resident = (long long)sms * kCtasPerSm;
    b->solo.assign(n, 0);
    for (int d = 0; d < n; ++d) {
        rc_plan_s* p = b->plans[d];
        const int n_lblk = first_block_only ? 1 : (b->nl[d] + LB - 1) / LB;
        long long least = -1;
        for (int i = 0; i < rcx::live_cascade_count(p); ++i) {
            const long long items = i == 0 ? (long long)p->nx * p->nz : p->lv[i].rays();
            const long long chunks = (items + G_rays - 1) / G_rays * n_lblk;
            least = least < 0 ? chunks : std::min(least, chunks);
        }
        b->solo[d] = least >= kSoloWaves * resident;
    }
    // per-cascade segment tables of the shared launches, chunks sorted by estimated cost (the
    // interval length a ray can actually march: min(b - a, domain diagonal) per chunk of rays)
    std::vector<LevelTables> T(C + 1);
    std::vector<rcx::LevelArgs> args((size_t)C * n);
    std::vector<rcx::PackArgs> pargs(n);
    for (int i = 0; i < C; ++i) {
        struct Seg { double cost; int d, lb; long long chunks; };
        std::vector<Seg> segs;
        for (int d = 0; d < n; ++d) {
            rc_plan_s* p = b->plans[d];
            args[(size_t)i * n + d] = rcx::level_args(p, i, b->nl[d], b->J[d], nullptr, nullptr, nullptr);
            if (b->solo[d]) continue;
            if (rcx::strips_for(p, i) > 1) continue;   // launched strip by strip after the batch
            const long long items = i == 0 ? (long long)p->nx * p->nz : p->lv[i].rays();
            const long long chunks = (items + G_rays - 1) / G_rays;
            const double diag = std::sqrt((double)p->nx * p->nx + (double)p->nz * p->nz);
            const double len = std::min(p->lv[i].b - p->lv[i].a, diag) * (i == 0 ? p->W0 : 1);
            const int n_lblk = first_block_only ? 1 : (b->nl[d] + LB - 1) / LB;
            for (int lb = 0; lb < n_lblk; ++lb) segs.push_back({len, d, lb, chunks});
        }
        std::stable_sort(segs.begin(), segs.end(), [](const Seg& x, const Seg& y) { return x.cost > y.cost; });
        for (const Seg& s : segs) {
            T[i].prefix.push_back(T[i].total);
            T[i].dom.push_back(s.d);
            T[i].lblk.push_back(s.lb);
            T[i].total += s.chunks;
        }
    }
    for (int d = 0; d < n; ++d) {
        rc_plan_s* p = b->plans[d];
        if (b->solo[d]) continue;
        pargs[d] = rcx::PackArgs{b->chi[d], b->eta[d], b->nl[d], 1, nullptr, nullptr,
                                 (long long)p->nx * p->nz, (float)p->voxel, p->d_packed,
                                 p->opt.precision != RC_STORE_F32 ? p->d_smax : nullptr};
        const long long chunks = ((long long)p->nx * p->nz + 255) / 256;
        const int n_lblk = first_block_only ? 1 : (b->nl[d] + LB - 1) / LB;
        for (int lb = 0; lb < n_lblk; ++lb) {
            T[C].prefix.push_back(T[C].total);
            T[C].dom.push_back(d);
            T[C].lblk.push_back(lb);
            T[C].total += chunks;
        }
    }
    // one device allocation for all tables
    size_t bytes = args.size() * sizeof(rcx::LevelArgs) + pargs.size() * sizeof(rcx::PackArgs);
    for (const auto& t : T) bytes += t.prefix.size() * (sizeof(long long) + 2 * sizeof(int)) + 64;
    bytes += 256;
    cudaError_t e = cudaMalloc(&b->d_tables, bytes);
    if (e != cudaSuccess) return bfail(RC_ERR_OOM, "rc_batch: table allocation");
    std::vector<unsigned char> host(bytes, 0);
    size_t off = 0;
    auto put = [&](const void* src, size_t nbytes) {
        off = (off + 15) & ~(size_t)15;
        const size_t at = off;
        std::copy((const unsigned char*)src, (const unsigned char*)src + nbytes, host.begin() + at);
        off += nbytes;
        return (unsigned char*)b->d_tables + at;
    };
    auto* d_args = (const rcx::LevelArgs*)put(args.data(), args.size() * sizeof(rcx::LevelArgs));
    auto* d_pargs = (const rcx::PackArgs*)put(pargs.data(), pargs.size() * sizeof(rcx::PackArgs));
    b->level.assign(C, {});
    for (int i = 0; i <= C; ++i) {
        auto* pre = (const long long*)put(T[i].prefix.data(), T[i].prefix.size() * sizeof(long long));
        auto* dom = (const int*)put(T[i].dom.data(), T[i].dom.size() * sizeof(int));
        auto* lbk = (const int*)put(T[i].lblk.data(), T[i].lblk.size() * sizeof(int));
        if (i < C) b->level[i] = {d_args + (size_t)i * n, pre, dom, lbk, (int)T[i].prefix.size(), T[i].total};
        else b->pack = {d_pargs, pre, dom, lbk, (int)T[i].prefix.size(), T[i].total};
    }
    if ((e = cudaMemcpy(b->d_tables, host.data(), bytes, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bcuda(e, "rc_batch: table upload");

    // cascade launches: one CTA per chunk, handed out in index order by the hardware
    b->grid.assign(C, 0);
    for (int i = 0; i < C; ++i) {
        int occ = 0;
        rcx::launch_batched_level(LB, b->VL, b->precision, i == 0, i < C - 1, b->level[i], 0,
                                  nullptr, &occ);
        if (occ < 1) return bfail(RC_ERR_UNSUPPORTED, "rc_batch: lane layout has no batched kernel");
        if (b->level[i].total > 0x7FFFFFFFLL)
            return bfail(RC_ERR_ARG, "rc_batch: more than 2^31 - 1 chunks in one cascade");
        b->grid[i] = (int)b->level[i].total;
    }
    b->pack_grid = (int)std::min<long long>(b->pack.total, (long long)sms * 8);

    // capture: [memset smax, pack] -> [scales] -> cascades top to bottom
    if (!b->cap && (e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return bcuda(e, "rc_batch: capture stream");
    if ((e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return bcuda(e, "rc_batch: begin capture");
    int launches = 0;
    const bool f16 = b->precision != RC_STORE_F32;
    cudaError_t le = cudaSuccess;
    rc_status sst = RC_OK;
    // the domains that fill the GPU alone, one after another, each with its own sequence
    for (int d = 0; d < n && sst == RC_OK; ++d) {
        if (!b->solo[d]) continue;
        rc_plan_s* p = b->plans[d];
        sst = rcx::solve_sequence(p, b->chi[d], b->eta[d],
                                  first_block_only ? std::min(b->nl[d], LB) : b->nl[d], b->J[d], b->cap);
        launches += p->last_launches;
    }
    if (sst != RC_OK) le = cudaErrorUnknown;
    const bool shared = b->pack.total > 0;
    if (f16 && shared)
        for (int d = 0; d < n && le == cudaSuccess; ++d) {
            if (b->solo[d]) continue;
            rc_plan_s* p = b->plans[d];
            le = cudaMemsetAsync(p->d_smax, 0, p->aux_count * sizeof(unsigned), b->cap);
        }
    if (le == cudaSuccess && shared) {
        le = rcx::launch_batched_pack(LB, b->pack, b->pack_grid, b->cap);
        ++launches;
    }
    if (f16 && shared)
        for (int d = 0; d < n && le == cudaSuccess; ++d) {
            if (b->solo[d]) continue;
            rc_plan_s* p = b->plans[d];
            le = rcx::launch_scales((b->nl[d] + LB - 1) / LB, p->d_smax, p->d_scale, b->cap);
            ++launches;
        }
    for (int i = C - 1; i >= 0 && le == cudaSuccess && shared; --i) {
        if (b->level[i].total > 0) {
            le = rcx::launch_batched_level(LB, b->VL, b->precision, i == 0, i < C - 1, b->level[i],
                                           b->grid[i], b->cap, nullptr);
            ++launches;
        }
        // domains whose cascade i is strip-split (large fields, long intervals): one launch
        // per wavelength block and strip, as in rc_formal_solve
        for (int d = 0; d < n && le == cudaSuccess; ++d) {
            rc_plan_s* p = b->plans[d];
            const int S = rcx::strips_for(p, i);
            if (S < 2 || b->solo[d]) continue;
            rcx::LevelArgs a = args[(size_t)i * n + d];
            a.it_state = p->d_it;
            a.n_strips = S;
            const int n_lblk = first_block_only ? 1 : (b->nl[d] + LB - 1) / LB;
            // as many wavelength blocks per launch as the plan's it_state holds
            const size_t per_blk = (size_t)a.rays * LB * sizeof(float2);
            const int G = std::max(1, std::min(n_lblk, (int)(p->it_bytes / per_blk)));
            for (int lb = 0; lb < n_lblk && le == cudaSuccess; lb += G)
                for (int ph = 0; ph < S && le == cudaSuccess; ++ph, ++launches) {
                    a.split_lb = lb;
                    a.split_nblk = std::min(G, n_lblk - lb);
                    a.phase = ph;
                    le = rcx::launch_level_split(LB, b->VL, b->precision, i < C - 1, a, b->cap);
                }
        }
    }
    e = cudaStreamEndCapture(b->cap, &b->graph);
    if (sst != RC_OK) return sst;
    if (le != cudaSuccess) return bcuda(le, "rc_batch: launch during capture");
    if (e != cudaSuccess) return bcuda(e, "rc_batch: end capture");
    if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess)
        return bcuda(e, "rc_batch: graph instantiate");
    b->launches = launches;
    return RC_OK;
}

}  // namespace

extern "C" {

rc_status rc_batch_create(int n, const rc_plan_t* plans, const float* const* chi,
                          const float* const* eta, const int* n_lambda, float* const* J,
                          int autotune, rc_batch_t* out) {
    rcx::set_last_error("");
    if (!out) return bfail(RC_ERR_ARG, "rc_batch_create: out is NULL");
    *out = nullptr;
    if (n < 1 || !plans || !chi || !eta || !n_lambda || !J)
        return bfail(RC_ERR_ARG, "rc_batch_create: n < 1 or NULL arrays");
    for (int d = 0; d < n; ++d) {
        if (!plans[d] || !chi[d] || !eta[d] || !J[d] || n_lambda[d] < 1)
            return bfail(RC_ERR_ARG, "rc_batch_create: NULL plan/buffer or n_lambda < 1 in domain " +
                                         std::to_string(d));
        if (plans[d]->sparse)
            return bfail(RC_ERR_UNSUPPORTED, "rc_batch_create: sparse plans are served by "
                                             "rc_formal_solve only");
        if (plans[d]->n_incl != 1)
            return bfail(RC_ERR_UNSUPPORTED, "rc_batch_create: inclinations are served by "
                                             "rc_formal_solve only");
        if (plans[d]->opt.bilinear_fix)
            return bfail(RC_ERR_UNSUPPORTED, "rc_batch_create: the bilinear fix is served by "
                                             "rc_formal_solve only");
        if (plans[d]->C != plans[0]->C || plans[d]->opt.precision != plans[0]->opt.precision ||
            plans[d]->device != plans[0]->device)
            return bfail(RC_ERR_ARG, "rc_batch_create: all plans need the same cascade count, "
                                     "storage precision and device");
        if ((n_lambda[d] + plans[d]->LB - 1) / plans[d]->LB > 65535)
            return bfail(RC_ERR_ARG, "rc_batch_create: too many wavelengths in a domain");
    }
    rc_batch_s* b = new (std::nothrow) rc_batch_s();
    if (!b) return bfail(RC_ERR_OOM, "rc_batch_create: host allocation");
    b->device = plans[0]->device;
    b->n = n;
    b->C = plans[0]->C;
    for (int d = 0; d < n; ++d) {
        b->plans.push_back(plans[d]);
        b->chi.push_back(chi[d]);
        b->eta.push_back(eta[d]);
        b->J.push_back(J[d]);
        b->nl.push_back(n_lambda[d]);
    }
    // every plan takes the first plan's lane layout (one kernel instantiation per cascade)
    for (int d = 1; d < n; ++d) {
        rc_status st = rcx::plan_set_layout(plans[d], plans[0]->LB, plans[0]->VL);
        if (st != RC_OK) {
            delete b;
            return st;
        }
    }
    rc_status st = RC_OK;
    if (autotune) {
        static const int cand[][2] = {{16, 4}, {8, 4}, {32, 4}, {8, 2}, {4, 4}};
        float best = INFINITY;
        int bLB = plans[0]->LB, bVL = plans[0]->VL;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        // each candidate is timed on the first lambda block of every domain and ranked by
        // time per wavelength slice
        for (const auto& c : cand) {
            for (int d = 0; d < n && st == RC_OK; ++d) st = rcx::plan_set_layout(plans[d], c[0], c[1]);
            if (st == RC_OK) st = build(b, true);
            if (st != RC_OK) break;
            long long slices = 0;
            for (int d = 0; d < n; ++d) slices += std::min(n_lambda[d], c[0]);
            cudaGraphLaunch(b->exec, b->cap);                   // warm-up
            cudaEventRecord(e0, b->cap);
            for (int r = 0; r < 2; ++r) cudaGraphLaunch(b->exec, b->cap);
            cudaEventRecord(e1, b->cap);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= (float)slices;
            if (ms < best) {
                best = ms;
                bLB = c[0];
                bVL = c[1];
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        for (int d = 0; d < n && st == RC_OK; ++d) st = rcx::plan_set_layout(plans[d], bLB, bVL);
    }
    if (st == RC_OK) st = build(b);
    if (st != RC_OK) {
        release(b);
        if (b->cap) cudaStreamDestroy(b->cap);
        delete b;
        return st;
    }
    *out = b;
    return RC_OK;
}

rc_status rc_batch_run(rc_batch_t b, void* stream) {
    rcx::set_last_error("");
    if (!b || !b->exec) return bfail(RC_ERR_ARG, "rc_batch_run: batch is NULL");
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? RC_OK : bcuda(e, "rc_batch_run");
}

rc_status rc_batch_info(rc_batch_t b, int* launches_per_run, int* lambda_block,
                        int* lambda_per_lane) {
    if (!b) return bfail(RC_ERR_ARG, "rc_batch_info: batch is NULL");
    if (launches_per_run) *launches_per_run = b->launches;
    if (lambda_block) *lambda_block = b->LB;
    if (lambda_per_lane) *lambda_per_lane = b->VL;
    return RC_OK;
}

int rc_batch_solo_domains(rc_batch_t b) {
    if (!b) return -1;
    return (int)std::count(b->solo.begin(), b->solo.end(), 1);
}

void rc_batch_destroy(rc_batch_t b) {
    if (!b) return;
    cudaDeviceSynchronize();
    release(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

rc_status rc_formal_solve_batched(int n, const rc_plan_t* plans, const float* const* chi,
                                  const float* const* eta, const int* n_lambda, float* const* J,
                                  void* stream) {
    rc_batch_t b = nullptr;
    rc_status st = rc_batch_create(n, plans, chi, eta, n_lambda, J, 0, &b);
    if (st != RC_OK) return st;
    st = rc_batch_run(b, stream);
    if (st == RC_OK) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) st = bcuda(e, "rc_formal_solve_batched");
    }
    rc_batch_destroy(b);
    return st;
}

}  // extern "C"
