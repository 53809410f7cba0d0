/*
 * rcx.h -- C ABI of librcx.so, the radiance-cascade (RC) formal solution of
 * Osborne & Sannikov, "Radiance Cascades: A Novel High-Resolution Formal
 * Solution for Multidimensional Non-LTE Radiative Transfer" (arXiv 2408.14425),
 * written for one NVIDIA B300 (sm_103a).
 *
 * Conventions shared by every entry point
 *   - Device pointers are plain CUDA device addresses on the device that was
 *     current when the plan was made.  Host pointers are ordinary (pageable
 *     or pinned) host memory.  The caller owns every buffer it passes in; the
 *     plan owns its scratch (packed fields, cascade storage, tables).
 *   - 2D arrays are row-major [nz][nx] with x fastest; per-wavelength arrays
 *     are [n_lambda][nz][nx].  Cell (ix, iz) covers [ix, ix+1] x [iz, iz+1]
 *     in voxel units.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream).  Only calls whose documentation says so
 *     synchronise.
 *   - Errors are returned as rc_status codes; nothing aborts or throws across
 *     the ABI.  rc_last_error() gives a one-line message for the calling
 *     thread's last failure.  A sticky CUDA error is reported as RC_ERR_CUDA.
 *   - A plan is not thread-safe: calls on one plan must not overlap in time
 *     (its scratch is shared by all of them).
 */
#ifndef RCX_H
#define RCX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rc_plan_s* rc_plan_t;

typedef enum {
    RC_OK = 0,
    RC_ERR_ARG = -1,           /* invalid argument (null pointer, bad size, unsupported value) */
    RC_ERR_OOM = -2,           /* device or host allocation failed */
    RC_ERR_CUDA = -3,          /* a CUDA runtime call failed (message in rc_last_error) */
    RC_ERR_TIMEOUT = -4,       /* a bounded device-side wait ran out */
    RC_ERR_NOT_CONVERGED = -5, /* an iteration hit its iteration cap */
    RC_ERR_UNSUPPORTED = -6    /* a valid request this build does not implement */
} rc_status;

/* Uniform 2D grid (Sec. 3.2: only uniform grids, traversed by DDA). */
typedef struct {
    int nx, nz;          /* cells per axis, >= 1 */
    double voxel_size;   /* physical edge length of a cell; chi is per this unit of length */
} rc_grid;

/* Storage precision of the merged radiance intervals between cascades. */
enum { RC_STORE_F32 = 0, RC_STORE_F16 = 1, RC_STORE_BF16 = 2 };

typedef struct {
    int precision;       /* RC_STORE_*: F16/BF16 store merged intervals with a per-cascade
                            scale and merge in FP32 (the ray march is always FP32) */
    int n_incl;          /* inclination rays per in-plane ray (2D invariance, Sec. 3.1); 1 = flatland */
    int interval_rule;   /* 0: interval lengths interval0 * 4^i, a_i = sum of the shorter ones;
                            1: a_i = interval0 * 4^(i-1), b_i = interval0 * 4^i (both satisfy Eq. 12-13) */
    int lambda_block;    /* wavelengths marched together along one ray (packed together per
                            voxel): 0 = default (16); 1, 2, 4, 8, 16 or 32 */
    int bilinear_fix;    /* 1: trace each cascade-i ray to the start of each of the four upper
                            probes' child rays before merging (Sec. 2.5); 0 = basic RC */
    int lambda_per_lane; /* wavelengths one GPU lane carries along its ray: 0 = default
                            (min(lambda_block, 4)); 1, 2, 4 or 8, at most lambda_block */
    int reserved[2];     /* must be zero */
} rc_options;

/* Fills *opt with the defaults (F32 storage, flatland, rule 0, automatic lane layout, basic RC). */
void rc_options_default(rc_options* opt);

/*
 * rc_plan -- geometry of a cascade set (Sec. 2.3, Eq. 12-13; Sec. 3.2).
 *   n_cascades  number of cascades C >= 1; the top one extends to the domain edge.
 *   dirs0       directions of cascade 0 (W_0 >= 1), directions theta_k = 2 pi (k+1/2)/W_0.
 *   branching   children per direction per cascade (2 alpha); this build supports 4 (alpha = 2,
 *               the value the paper uses throughout, Sec. 2.4).
 *   interval0   length of the cascade-0 interval in voxels (> 0).
 *   opt         NULL for defaults.
 * Cascade i has probes at ((k+1/2) 2^i, (m+1/2) 2^i), ceil(n/2^i) per axis, W_0 4^i directions,
 * and the interval [a_i, b_i] of interval_rule.  The plan copies its direction tables to the
 * current device (one small allocation); scratch for the solves is allocated on first use or by
 * rc_plan_reserve.  On success *out owns the plan (free with rc_plan_destroy).
 * Errors: RC_ERR_ARG (bad sizes, NULL out), RC_ERR_UNSUPPORTED (branching != 4),
 * RC_ERR_OOM, RC_ERR_CUDA.
 */
rc_status rc_plan(const rc_grid* grid, int n_cascades, int dirs0, int branching,
                  float interval0, const rc_options* opt, rc_plan_t* out);

/* Releases a plan and its device memory (synchronises the device first).  NULL is a no-op. */
void rc_plan_destroy(rc_plan_t plan);

/* Grows the plan's scratch so that solves of up to n_lambda wavelengths allocate nothing
 * (needed before capturing a solve in a CUDA graph).  Synchronous.
 * Errors: RC_ERR_ARG, RC_ERR_OOM, RC_ERR_CUDA. */
rc_status rc_plan_reserve(rc_plan_t plan, int n_lambda);

/* Bytes of device scratch the plan holds now. */
size_t rc_plan_scratch_bytes(rc_plan_t plan);

/*
 * rc_formal_solve -- J for every wavelength (GivenFs mode, Sec. 3.8).
 *   chi, eta   device, FP32 [n_lambda][nz][nx]: opacity (per voxel_size length) and
 *              emissivity, both >= 0.  Isotropic (no velocity field).
 *   J          device, FP32 [n_lambda][nz][nx], written: mean intensity of Eq. 1 at every
 *              cell centre (the cascade-0 probes), as the equal-weight mean over the W_0
 *              merged cascade-0 rays (flatland) or over W_0 x n_incl rays.
 *   alo        device FP32 [n_lambda][nz][nx] or NULL: angle-mean diagonal operator
 *              (1/W_0) sum_k (1 - exp(-chi d_k)), d_k the path from the cell centre to its edge
 *              along direction k (Eq. 17; the exponent form printed there is read as the
 *              local operator of the piecewise-constant update, Eq. 16).
 * Each interval is marched through the voxels it crosses with Eq. 16 (FP32), merged with
 * the child-cone average of the bilinearly interpolated upper cascade (Sec. 2.3.1, Eq. 11,
 * the nearer interval attenuating the farther), with the lookup clamped at the edges
 * (Sec. 2.5); outside the domain there is free space (Sec. 3.4).
 * Opacities below 1e-30 per voxel are raised to 1e-30 (the emission eta ds of such a cell is
 * kept).  Asynchronous on `stream`; may allocate scratch on first use (see rc_plan_reserve).
 * Errors: RC_ERR_ARG (NULL pointers, n_lambda < 0), RC_ERR_OOM, RC_ERR_CUDA.
 */
rc_status rc_formal_solve(rc_plan_t plan, const float* chi, const float* eta, int n_lambda,
                          float* J, float* alo, void* stream);

/*
 * rc_formal_solve_host -- as rc_formal_solve, with chi, eta, J (and alo) in HOST memory.
 * The wavelengths are processed in chunks; each chunk's host-to-device copies, solve and
 * device-to-host copy of J are pipelined on two internal streams.  Pinned host buffers
 * copy fastest.  Synchronous: returns when J is in host memory.
 * Errors: as rc_formal_solve.
 */
rc_status rc_formal_solve_host(rc_plan_t plan, const float* chi_host, const float* eta_host,
                               int n_lambda, float* J_host, float* alo_host);

/* Per-cascade geometry of a plan: probes per axis, directions, interval bounds (b = inf for
 * the top cascade).  Any output pointer may be NULL.  Errors: RC_ERR_ARG. */
rc_status rc_plan_cascade(rc_plan_t plan, int i, int* px, int* pz, long long* dirs,
                          double* a, double* b);

/* Number of device kernels the last rc_formal_solve(_host) on this plan launched. */
int rc_plan_last_launch_count(rc_plan_t plan);

/*
 * Per-launch timing (tracing).  With timing enabled, rc_formal_solve records a CUDA event on
 * its stream before its first launch and after each launch.  rc_plan_launch_times then waits
 * for the last solve's events and writes up to max_n durations in milliseconds, in launch
 * order, and the count to *n_out; rc_plan_launch_name gives the kernel name of launch i
 * ("pack", "scale", "cascade <i>").  The host-buffer entry point records nothing.
 * Errors: RC_ERR_ARG (NULL plan/outputs, timing off or no timed solve yet), RC_ERR_CUDA.
 */
rc_status rc_plan_set_timing(rc_plan_t plan, int enable);
rc_status rc_plan_launch_times(rc_plan_t plan, float* ms_out, int max_n, int* n_out);
const char* rc_plan_launch_name(rc_plan_t plan, int i);

/*
 * rc_formal_solve_noalloc -- the formal solution of rc_formal_solve without any device
 * allocation, for callers that cannot call cudaMalloc: code whose device memory is owned by
 * another allocator (a framework's caching pool, a memory budget fixed up front), code that
 * runs where allocation is not allowed or would synchronise the device, and embedders that
 * must not grow the process's device footprint after start-up.  The paper has no counterpart;
 * it is a deployment variant of rc_formal_solve.
 *   grid, n_cascades, dirs0, interval0   as rc_plan, with branching 4, interval_rule 0,
 *                                        FP32 interval storage, 4-wavelength blocks and
 *                                        2 wavelengths per lane.
 *   chi, eta, n_lambda, J, alo, stream   as rc_formal_solve (caller-owned device buffers).
 * Scratch: a static device array of 32 MiB (33554432 bytes) inside librcx.so, which every GPU
 * that loads the library holds until the process exits.  It must hold the direction tables,
 * the packed field (n_lambda rounded up to 4) x nx x nz x 8 bytes and two cascades of merged
 * intervals (rounded n_lambda x the largest cascade's rays x 4 bytes each), each rounded up to
 * 256 bytes; for example 256 x 256 with 8 wavelengths and 7 cascades fits.  A larger problem
 * is rejected with RC_ERR_ARG and a message giving the bytes it needs.
 * The first call on a device (with that device current) looks up the array's device address
 * once with cudaGetSymbolAddress; make that first call before any stream capture.
 * All calls share the one array, and it keeps the last call's contents: every call rewrites
 * what it reads, so nothing has to be cleared, but calls whose work overlaps on the GPU (on
 * different streams, or from several host threads) race on the array and must be serialised
 * by the caller.  Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * Errors: RC_ERR_ARG (bad sizes, NULL pointers, problem too large), RC_ERR_CUDA.
 */
rc_status rc_formal_solve_noalloc(const rc_grid* grid, int n_cascades, int dirs0, float interval0,
                                  const float* chi, const float* eta, int n_lambda, float* J,
                                  float* alo, void* stream);

/* One-line message for the calling thread's last error ("" if none). */
const char* rc_last_error(void);

/* Static name of a status code. */
const char* rc_status_string(rc_status s);

#ifdef __cplusplus
}
#endif

#endif /* RCX_H */
