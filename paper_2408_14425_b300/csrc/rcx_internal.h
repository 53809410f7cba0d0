// rcx_internal.h -- plan layout and kernel launch arguments shared by the host
// side (rcx_plan.cu) and the kernels (rcx_fs_kernels.cu) of librcx.so.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/rcx.h"

namespace rcx {

// Opacities below this (per voxel) are raised to it; the cell's emission eta ds
// survives through the source function eta / chi.
constexpr float kChiFloor = 1e-30f;
// Warps per CTA of the march kernels.  4 (at 12 resident CTAs/SM, 40 registers) measured
// 824-827 slices/s at 1024^2 x 64 wavelengths against 795, 793, 785, 797 and 810 with 2, 3,
// 5, 6 and 8 (same 40 registers, 45-48 warps per SM): a CTA keeps its slot until its
// slowest warp ends, and smaller CTAs waste less of it.
#ifndef RCX_WARPS_PER_CTA
#define RCX_WARPS_PER_CTA 4
#endif
constexpr int kWarpsPerCta = RCX_WARPS_PER_CTA;
// Merged-interval scale for 16-bit storage: values are stored as R / (S_max 2^-14),
// which keeps every merged interval (R <= S_max in free space) below 2^14.
constexpr float kF16Headroom = 16384.0f;

struct LevelGeom {
    int Px = 0, Pz = 0;      // probes per axis
    long long W = 0;         // directions
    double a = 0, b = 0;     // interval [a, b] in voxels (b = inf on the top cascade)
    long long rays() const { return (long long)Px * Pz * W; }
};

// Arguments of one cascade-level launch (passed by value).
struct LevelArgs {
    const float2* field;     // packed (chi per voxel, S) [n_lblk][ncell][LB]
    long long ncell;
    int nx, nz;
    int Px, Pz;              // this cascade's probes per axis
    int W;                   // this cascade's directions
    int Wshift;              // log2(W) if W is a power of two, else -1
    float spacing;           // probe spacing 2^i (voxels)
    float a, b;              // interval (b = +inf on the top cascade)
    float a_up;              // start of the upper cascade's interval (bilinear fix)
    int bilinear_fix;        // 1: trace to the upper probes' child starts (Sec. 2.5)
    const float2* dirs;      // W unit vectors (cos, sin)
    long long rays;          // Px * Pz * W
    // upper cascade (merged), NULL on the top cascade
    const void* R_up;
    int Px_up, Pz_up;
    long long R_up_lstride;  // elements per lambda block in R_up
    // this cascade's merged output (levels >= 1)
    void* R_out;
    long long R_out_lstride;
    const float* scale;      // per lambda block storage scale (16-bit storage), NULL = 1
    // cascade 0 outputs
    const int* probe_list;   // sparse: flagged probes of this cascade (ascending), else NULL
    float* J;
    float* alo;
    float* J_eff;            // J without the cell's own segment emission (MALI), may be NULL
    float* alo_c;            // 1 - alo, may be NULL
    int n_lambda;
    int max_steps;           // upper bound on cells crossed by one ray (nx + nz + 2)
    // strip-split march (launch_level_split): partial (I, T) of every ray of one lambda
    // block [block][ray][LB], the strip count, this launch's phase, its first lambda block
    // and block count (0 counts as 1), and the strip's columns [strip_x0, strip_x1) (set by
    // launch_level_split)
    float2* it_state;
    int n_strips, phase, split_lb, split_nblk;
    int strip_x0, strip_x1;
};

struct PackArgs {
    const float* chi;
    const float* eta;
    int n_lambda;            // physical wavelengths
    int n_incl;              // inclinations per wavelength (virtual wavelength l n_incl + j)
    const float* incl_r;     // 1/sqrt(1 - mu_j^2) per inclination (NULL when n_incl == 1)
    const unsigned char* active;  // sparse: inactive cells packed transparent (NULL = all)
    long long ncell;
    float voxel;
    float2* out;
    unsigned int* smax_bits;  // per lambda block, may be NULL
};

// Emergent intensity along caller rays (front to back, Sec. 3.9).
struct EmergentArgs {
    const float2* field;
    long long ncell;
    int nx, nz;
    const float* rays;            // [n_rays][4]: ox, oz, wx, wz (voxels)
    long long n_rays;
    float* I;                     // [n_lambda][n_rays]
    float* contrib;               // [n_lambda][ncell] or NULL
    int n_lambda;
    int max_steps;
};

// A batch launch: CTA-sized chunks of all (domain, lambda block) segments of one cascade.
struct BatchLevelArgs {
    const LevelArgs* args;        // per domain (device)
    const long long* prefix;      // first chunk of each segment (device), ascending
    const int* seg_domain;        // domain of each segment (device)
    const int* seg_lblk;          // lambda block of each segment (device)
    int n_seg;
    long long total;              // chunks in all segments
};

struct BatchPackArgs {
    const PackArgs* args;
    const long long* prefix;
    const int* seg_domain;
    const int* seg_lblk;
    int n_seg;
    long long total;
};

// Sparse flags (Sec. 3.5): seed cascade 0 from the cell mask, propagate each flagged
// probe to the upper probes its bilinear lookup brackets, and compact the flagged probes
// of a cascade into an ascending list (count -> *n_out, device).
cudaError_t launch_flags_seed(const unsigned char* active, unsigned char* f0, long long ncell,
                              cudaStream_t s);
cudaError_t launch_flags_up(const unsigned char* f, int Px, int Pz, unsigned char* fu, int Pxu,
                            int Pzu, cudaStream_t s);
cudaError_t launch_compact(const unsigned char* f, long long n, int* list, int* n_out,
                           cudaStream_t s);

cudaError_t launch_emergent(int LB, int n_lblk, const EmergentArgs& a, cudaStream_t s);

// Weighted sum over inclinations: out[l][c] = sum_j w_j in[l n_incl + j][c].
cudaError_t launch_incl_reduce(const float* in, float* out, int n_lambda, int n_incl,
                               const float* w, long long ncell, cudaStream_t s);

// Launchers (rcx_fs_kernels.cu).  Return the CUDA launch error.
// With occ != NULL the batched launcher only reports the kernel's resident CTAs per SM.
cudaError_t launch_batched_level(int LB, int VL, int precision, bool level0, bool has_up,
                                 const BatchLevelArgs& b, int grid, cudaStream_t s, int* occ);
cudaError_t launch_batched_pack(int LB, const BatchPackArgs& b, int grid, cudaStream_t s);
cudaError_t launch_pack(int LB, int n_lblk, const PackArgs& a, cudaStream_t s);
// One phase of a strip-split cascade (cascades >= 1, no bilinear fix): lambda block
// a.split_lb, the rays' pieces inside strip a.phase (or its mirror for rays moving to -x).
cudaError_t launch_level_split(int LB, int VL, int precision, bool has_up, const LevelArgs& a,
                               cudaStream_t s);
bool level_split_supported(int LB, int VL);
cudaError_t launch_level(int LB, int VL, int precision, bool level0, bool has_up, int n_lblk,
                         const LevelArgs& a, cudaStream_t s);
// The highest launched cascade (no upper) over a list of CTAs: flags[c] = 1 (flags zeroed
// by the caller) for every CTA c of per_cta consecutive rays holding a ray whose interval
// comes within one voxel of the box (FP64, so a CTA left out has no ray that the FP32
// march can enter the box with); then launch_level over the n_cta listed CTAs only
// (lane-group march, a.Wshift >= 0, no sparse list, no bilinear fix).
cudaError_t launch_top_hits(const LevelArgs& a, int per_cta, unsigned char* flags,
                            cudaStream_t s);
bool level_list_supported(int LB, int VL, const LevelArgs& a);
cudaError_t launch_level_list(int LB, int VL, int precision, int n_lblk, const LevelArgs& a,
                              const int* cta_list, long long n_cta, cudaStream_t s);
// The shared-DDA march of a cascade >= 1 (one warp walks the DDA of 32 rays into shared
// memory and replays it for their wavelengths): whether a launch can take it, the unsplit
// launch and one phase of a strip-split cascade (arguments as launch_level(_split)).
bool level_sdda_supported(int LB, int VL, const LevelArgs& a);
cudaError_t launch_level_sdda(int LB, int VL, int precision, bool has_up, int n_lblk,
                              const LevelArgs& a, cudaStream_t s);
cudaError_t launch_level_split_sdda(int LB, int VL, int precision, bool has_up,
                                    const LevelArgs& a, cudaStream_t s);
cudaError_t launch_scales(int n_lblk, const unsigned int* smax_bits, float* scale,
                          cudaStream_t s);

// Sets the calling thread's rc_last_error() message (rcx_plan.cu).
void set_last_error(const std::string& msg);

}  // namespace rcx

struct rc_plan_s;
namespace rcx {
// Launch arguments of cascade i of a plan whose scratch holds n_lambda (rcx_plan.cu).
LevelArgs level_args(const rc_plan_s* p, int i, int n_lambda, float* J, float* alo,
                     float* J_eff, float* alo_c);
rc_status plan_reserve(rc_plan_s* p, int n_lambda);
// Guard band on each side of a packed field of nx-wide rows and LB wavelengths per voxel:
// one row plus one voxel, so the march's one-step-ahead fetch past the exit face stays in
// the allocation.  Rounded to 256 bytes.
inline size_t packed_guard_bytes(int nx, int LB) {
    return (((size_t)(nx + 1) * LB * 2 * sizeof(float)) + 255) & ~(size_t)255;
}
// strips of the strip-split march of cascade i of a plan (1 = not split)
int strips_for(const rc_plan_s* p, int i);
// cascades 0 .. live-1 of a plan can be non-zero (the rest lie in free space)
int live_cascade_count(const rc_plan_s* p);
// the launch sequence of rc_formal_solve (J only) on stream s, without its timing events;
// the plan's scratch must already hold n_lambda (nothing is allocated, so it may be captured)
rc_status solve_sequence(rc_plan_s* p, const float* chi, const float* eta, int n_lambda, float* J,
                         cudaStream_t s);
rc_status plan_set_layout(rc_plan_s* p, int LB, int VL);
// Device tables of an atom's levels: E/k [K] and g (rcx_nlte.cu).
rc_status atom_levels(rc_atom_t a, const double** Ek, const double** g, int* nlev,
                      int* n_per_line, int* n_lines);
}  // namespace rcx

struct rc_plan_s {
    int device = 0;
    int nx = 0, nz = 0;
    double voxel = 1.0;
    int C = 0, W0 = 0, B = 0;
    float L0 = 1.0f;
    rc_options opt{};
    int LB = 4;                      // wavelengths per lane group (one ray)
    int VL = 1;                      // wavelengths per lane
    int march = RC_MARCH_SHARED_DDA; // cascades >= 1: shared-DDA march where it applies
    unsigned march_tuned = 0;        // RC_MARCH_TUNED: bit i = cascade i takes the shared DDA
    int n_incl = 1;                  // inclination quadrature (2D invariance)
    float* d_incl = nullptr;         // [r_j (n_incl)][w_j (n_incl)]
    float* d_vout = nullptr;         // per-inclination cascade-0 outputs before the reduction
    size_t vout_floats = 0;
    // sparsity (Sec. 3.5): flags and flagged-probe lists per cascade, or none
    bool sparse = false;
    unsigned char* d_active = nullptr;     // copy of the cell mask
    void* d_sparse = nullptr;              // flags and lists of every cascade
    std::vector<const int*> probe_list;    // per cascade
    std::vector<long long> n_flagged;      // per cascade
    std::vector<rcx::LevelGeom> lv;
    // The highest launched cascade has no upper cascade, so a ray that misses the domain
    // stores 0.  Where most of its CTAs hold only such rays (long intervals from probes
    // near the edges), the solve clears its output and launches the listed CTAs alone.
    int* d_top_list = nullptr;       // CTAs with a ray that can reach the box, ascending
    long long top_hits = -1;         // their count; -1: no list (launch every CTA)
    int top_cascade = -1;            // the cascade the list is for
    int top_per_cta = 0;             // rays per CTA the list was made for
    bool top_list_on = true;         // rc_plan_set_top_list
    std::vector<size_t> dir_off;     // offset of each cascade's table in d_dirs
    float2* d_dirs = nullptr;
    // scratch
    float2* d_packed = nullptr;        // inside d_packed_raw, after a guard band
    float2* d_packed_raw = nullptr;
    size_t packed_guard = 0;           // bytes of guard band on each side of the field
    float2* d_it = nullptr;            // partial (I, T) of a strip-split cascade, one lambda block
    size_t it_bytes = 0;
    size_t packed_bytes = 0;
    void* d_R[2] = {nullptr, nullptr};
    size_t R_bytes = 0;              // bytes of each of the two cascade buffers
    unsigned int* d_smax = nullptr;  // per lambda block max source function (bits)
    float* d_scale = nullptr;
    size_t aux_count = 0;            // lambda blocks the smax/scale arrays hold
    int cap_lambda = 0;              // largest n_lambda the scratch holds
    // host-buffer pipeline
    cudaStream_t s_io[3] = {nullptr, nullptr, nullptr};   // copies in, solves, copies out
    float* d_stage = nullptr;        // 2 chunks x (chi, eta, J, alo)
    size_t stage_bytes = 0;
    cudaEvent_t io_done[2] = {nullptr, nullptr};   // staging buffer b free (its J copied out)
    long long io_chunks = 0;         // chunks enqueued so far (buffer of a chunk: count % 2)
    int last_launches = 0;
    // tracing
    bool timing = false;
    std::vector<cudaEvent_t> ev;     // ev[0] before the first launch, ev[j+1] after launch j
    std::vector<std::string> launch_names;
    int timed_launches = 0;
};
