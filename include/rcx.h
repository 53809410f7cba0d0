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
    RC_ERR_UNSUPPORTED = -6    /* a valid request the library does not implement */
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
    int n_incl;          /* inclination rays per in-plane ray (2D invariance, Sec. 3.1): 1 = flatland,
                            up to 16.  Gauss-Radau nodes in mu = cos(angle to the invariant axis)
                            on [0, 1) with the fixed node at the in-plane ray; each inclination
                            marches the same x-z path with chi and eta scaled by
                            1/sqrt(1 - mu^2); J, alo, J_eff, alo_c are their weighted sum.
                            Costs n_incl times the flatland work; not in batches. */
    int interval_rule;   /* 0: interval lengths interval0 * 4^i, a_i = sum of the shorter ones;
                            1: a_i = interval0 * 4^(i-1), b_i = interval0 * 4^i (both satisfy Eq. 12-13) */
    int lambda_block;    /* wavelengths marched together along one ray (packed together per
                            voxel): 0 = default (16); 1, 2, 4, 8, 16 or 32 */
    int bilinear_fix;    /* 1: trace each cascade-i ray to the start of each of the four upper
                            probes' child rays before merging (Sec. 2.5; 4x the rays below the
                            top cascade); serves J only (rc_formal_solve with alo = NULL,
                            not the MALI outputs or batches); 0 = basic RC */
    int lambda_per_lane; /* wavelengths one GPU lane carries along its ray: 0 = default
                            (min(lambda_block, 4)); 1, 2, 4 or 8, at most lambda_block */
    int strips;          /* strip-split march of long-ray cascades: 0 = automatic (a cascade
                            whose intervals reach half the domain, when one wavelength block
                            of the packed field exceeds 96 MiB, runs as one launch per
                            vertical strip of about 64 MiB per wavelength block, so each
                            launch gathers from a strip that stays in L2); 1 = never; 2..16 =
                            that many strips on every cascade >= 1.  Results agree with the
                            unsplit march to FP32 rounding.  Not with the bilinear fix; lane
                            layouts with 4 wavelengths per lane and 8-32 per ray.  The strips
                            hand a partial (I, T) per ray and wavelength (8 bytes) from one
                            launch to the next; one launch covers as many wavelength blocks as
                            fit 8 GiB of that state, and the plan's scratch holds it. */
    int reserved;        /* must be zero */
} rc_options;

/* Fills *opt with the defaults (F32 storage, flatland, rule 0, automatic lane layout, basic RC). */
void rc_options_default(rc_options* opt);

/*
 * rc_plan -- geometry of a cascade set (Sec. 2.3, Eq. 12-13; Sec. 3.2).
 *   n_cascades  number of cascades C >= 1; the top one extends to the domain edge.
 *   dirs0       directions of cascade 0 (W_0 >= 1), directions theta_k = 2 pi (k+1/2)/W_0.
 *   branching   children per direction per cascade (2 alpha); the library supports 4 (alpha = 2,
 *               the value the paper uses throughout, Sec. 2.4).
 *   interval0   length of the cascade-0 interval in voxels (> 0).
 *   opt         NULL for defaults.
 * Cascade i has probes at ((k+1/2) 2^i, (m+1/2) 2^i), ceil(n/2^i) per axis, W_0 4^i directions,
 * and the interval [a_i, b_i] of interval_rule.  The plan copies its direction tables to the
 * current device (one small allocation) and lists the CTAs of its highest launched cascade
 * that can reach the domain (rc_plan_set_top_list: two small kernels on the default stream
 * and a read-back, so creation is synchronous); scratch for the solves is allocated on first
 * use or by rc_plan_reserve.  On success *out owns the plan (free with rc_plan_destroy).
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

/* Bytes of device scratch the plan holds now: packed field with its guard bands, two
 * cascades of merged intervals, the strips' partial state (at most 8 GiB) and per-block
 * scales, plus the host entry's staging buffers once it has run. */
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
 * (Sec. 2.5); outside the domain there is free space (Sec. 3.4).  Top cascades whose
 * intervals all start beyond the farthest domain corner from each of their probes are
 * identically zero and are not launched (without the bilinear fix).
 * Opacities below 1e-30 per voxel are raised to 1e-30 (the emission eta ds of such a cell is
 * kept).  Asynchronous on `stream`; may allocate scratch on first use (see rc_plan_reserve).
 * Errors: RC_ERR_ARG (NULL pointers, n_lambda < 0), RC_ERR_OOM, RC_ERR_CUDA.
 */
rc_status rc_formal_solve(rc_plan_t plan, const float* chi, const float* eta, int n_lambda,
                          float* J, float* alo, void* stream);

/*
 * rc_formal_solve_host -- as rc_formal_solve, with chi, eta, J (and alo) in HOST memory.
 * The wavelengths are processed in chunks; each chunk's host-to-device copies, solve and
 * device-to-host copy of J run on three internal streams, so a chunk's copies overlap its
 * neighbours' solves.  Pinned host buffers
 * copy fastest.  Synchronous: returns when J is in host memory.
 * Errors: as rc_formal_solve.
 */
rc_status rc_formal_solve_host(rc_plan_t plan, const float* chi_host, const float* eta_host,
                               int n_lambda, float* J_host, float* alo_host);

/*
 * rc_formal_solve_host_async -- rc_formal_solve_host without the wait at the end (a
 * deployment variant with no counterpart in the paper; the solve itself is rc_formal_solve's):
 * the copies and solves are enqueued on the plan's three streams and the call returns.  Consecutive calls
 * on one plan pipeline: a call's first chunk is copied in while the previous call's last chunk
 * is solved, and the previous call's last J is copied out while this call's first chunk is
 * solved (the staging buffers alternate across calls); chunks are whole wavelength blocks of
 * up to 64 wavelengths (one solve per call at 64 wavelengths and 16 per block).  The host buffers of a call must stay
 * valid, and chi / eta unmodified, until the call has completed: after rc_plan_wait, or after
 * a later rc_formal_solve_host on the same plan returns.  Until then the plan must not be used
 * by other calls on other streams (rc_formal_solve and friends share its scratch).
 * rc_plan_wait -- blocks until every host-buffer solve enqueued on the plan has completed and
 * its results are in host memory.
 * Errors: as rc_formal_solve_host; asynchronous CUDA errors are reported by rc_plan_wait.
 */
rc_status rc_formal_solve_host_async(rc_plan_t plan, const float* chi, const float* eta,
                                     int n_lambda, float* J, float* alo);
rc_status rc_plan_wait(rc_plan_t plan);

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
 * once with cudaGetSymbolAddress; make that first call before any stream capture.  The address
 * is kept together with the ID of the CUDA context it came from: after cudaDeviceReset (or
 * when the primary context is released and created again) the module is loaded anew and the
 * array may move, so the next call finds a different context, looks the address up again
 * (that call is again a first call) and never launches on the old address.
 * All calls share the one array, and it keeps the last call's contents: every call rewrites
 * what it reads, so nothing has to be cleared, but calls whose work overlaps on the GPU (on
 * different streams, or from several host threads) race on the array and must be serialised
 * by the caller.  Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * Errors: RC_ERR_ARG (bad sizes, NULL pointers, problem too large), RC_ERR_CUDA.
 */
rc_status rc_formal_solve_noalloc(const rc_grid* grid, int n_cascades, int dirs0, float interval0,
                                  const float* chi, const float* eta, int n_lambda, float* J,
                                  float* alo, void* stream);

/*
 * Sparsity (Sec. 3.5): restrict the plan to the cells with active[c] != 0 (device uint8
 * [nz][nx]; NULL restores the dense plan).  Inactive cells are transparent with no emission;
 * the cascade-0 probes of active cells are flagged, every flagged probe flags the upper probes
 * its bilinear lookup brackets (up to the top cascade), and the cascade kernels run the flagged
 * probes only (flags and the ascending probe lists are built on the device).  Solves then
 * write J (alo, J_eff, alo_c) = 0 for inactive cells, and rc_nlte_solve keeps their
 * populations.  Synchronous.  Not for batches.  Errors: RC_ERR_ARG, RC_ERR_OOM, RC_ERR_CUDA.
 */
rc_status rc_plan_set_active(rc_plan_t plan, const unsigned char* active, void* stream);
/* Flagged probes per cascade (all probes for a dense plan); per_cascade has n_cascades entries. */
rc_status rc_plan_active_probes(rc_plan_t plan, long long* per_cascade);

/* Lane layout of a plan's march: wavelengths per ray (packed together per voxel) and per GPU
 * lane; see rc_options.  Changing lambda_block re-allocates the plan's scratch (synchronous).
 * Errors: RC_ERR_ARG, RC_ERR_OOM, RC_ERR_CUDA. */
rc_status rc_plan_set_lane_layout(rc_plan_t plan, int lambda_block, int lambda_per_lane);
rc_status rc_plan_get_lane_layout(rc_plan_t plan, int* lambda_block, int* lambda_per_lane);

/*
 * How the cascades >= 1 walk their rays (the DDA of Sec. 3.2 through the uniform voxel grid;
 * no counterpart choice in the paper, whose DexRT walks each ray in its own thread).
 *   RC_MARCH_LANE_GROUP  every lane of a ray's lane group walks the ray's DDA itself.
 *   RC_MARCH_SHARED_DDA  (default) the cascades whose intervals are at most 16 voxels long
 *                        take the shared-DDA march: a warp owns 32 rays, each lane walks one
 *                        ray's DDA for a chunk of steps into shared memory, and the warp
 *                        replays the chunk for the rays' wavelengths (one DDA walk per 32 rays
 *                        instead of per 8); longer cascades keep the lane-group march, which is
 *                        faster there (its 8 rays per warp keep more gathers in flight and a
 *                        smaller L2 working set).
 *   RC_MARCH_SHARED_DDA_ALL  the shared-DDA march on every cascade >= 1 (for comparison).
 * The shared-DDA march applies to dense plans with a power-of-two direction count, the 16 x 4
 * lane layout and no bilinear fix; other plans keep the lane-group march.  All modes give
 * identical results.  Takes effect at the next solve.  Errors: RC_ERR_ARG.
 */
enum { RC_MARCH_LANE_GROUP = 0, RC_MARCH_SHARED_DDA = 1, RC_MARCH_SHARED_DDA_ALL = 2,
       RC_MARCH_TUNED = 3 };
rc_status rc_plan_set_march(rc_plan_t plan, int mode);
rc_status rc_plan_get_march(rc_plan_t plan, int* mode);
/* Bit i of *mask set: cascade i takes the shared-DDA march under the plan's current mode.
 * RC_MARCH_TUNED is set by rc_plan_autotune (a per-cascade choice by timing); setting another
 * mode with rc_plan_set_march discards it.  Errors: RC_ERR_ARG. */
rc_status rc_plan_get_march_cascades(rc_plan_t plan, unsigned* mask);

/*
 * The highest launched cascade has no cascade above it (those above lie in free space,
 * Sec. 3.4), so a ray whose interval misses the domain has R = 0 there.  At creation a
 * plan lists the CTAs of that cascade holding a ray whose interval comes within one voxel
 * of the box (an FP64 test, conservative against the FP32 march); when the list leaves
 * out at least half of them, each solve clears the cascade's merged intervals and marches
 * the listed CTAs alone.  The result is bit-identical to marching every CTA.  The list
 * serves the default lane layout (16 wavelengths per ray, 4 per lane) with the lane-group
 * march on a dense plan without the bilinear fix; any other solve marches every CTA.
 * rc_plan_set_top_list(plan, 0) turns it off, (plan, 1) back on (the default).
 * rc_plan_get_top_list reports the cascade (-1: no list), the listed CTAs and the CTAs of
 * that cascade (any pointer may be NULL).  Errors: RC_ERR_ARG.
 */
rc_status rc_plan_set_top_list(rc_plan_t plan, int enable);
rc_status rc_plan_get_top_list(rc_plan_t plan, int* cascade, long long* listed,
                               long long* total);

/*
 * rc_plan_autotune -- times the formal solution of these inputs (device buffers as
 * rc_formal_solve; J is overwritten) with each candidate lane layout (16/4, 8/4, 32/4, 8/2,
 * 4/4, 4/2, 4/1, 2/2, 1/1 wavelengths per ray / per lane; blocks wider than twice n_lambda
 * skipped), keeps the fastest on the plan and reports it.  Then, unless the plan's march is
 * RC_MARCH_LANE_GROUP, it times every cascade with both marches and keeps the faster per
 * cascade (mode RC_MARCH_TUNED; rc_plan_get_march_cascades reports the choice).  Synchronous.
 * Errors: RC_ERR_ARG, RC_ERR_OOM, RC_ERR_CUDA.
 */
rc_status rc_plan_autotune(rc_plan_t plan, const float* chi, const float* eta, int n_lambda,
                           float* J, void* stream, int* lambda_block, int* lambda_per_lane);

/*
 * Batched formal solutions (independent problems solved together, Sec. 3.6: wavelengths and
 * domains are independent).  A batch binds n plans (same n_cascades, storage precision and
 * device; every plan is switched to the first plan's lane layout) to fixed device buffers
 * chi[d], eta[d], J[d] ([n_lambda[d]][nz_d][nx_d]).  A domain large enough to fill the GPU
 * on its own (at least 4 waves of CTAs, counted at 12 per SM, in every cascade that is not in
 * free space) keeps its own launch sequence, that of rc_formal_solve.  For the other
 * domains each cascade is ONE launch over a work list of CTA-sized chunks of every (domain,
 * wavelength block), sorted by estimated cost (interval length a ray can march, longest
 * first), one chunk per CTA; packing is one launch for all of them.  The whole sequence is
 * captured once into a CUDA graph; rc_batch_run
 * replays it on `stream` (asynchronous).  With autotune != 0 creation times graph replays of
 * the candidate lane layouts (16/4, 8/4, 32/4, 8/2, 4/4) on the first wavelength block of
 * every bound domain, ranks them by time per wavelength slice and keeps the fastest.
 * Scratch is reserved at creation, so runs allocate nothing.  The buffers must outlive the
 * batch; a batch must not run concurrently with another use of its plans.
 * Errors: RC_ERR_ARG (mismatched plans, NULL buffers), RC_ERR_OOM, RC_ERR_CUDA.
 */
typedef struct rc_batch_s* rc_batch_t;
rc_status rc_batch_create(int n, const rc_plan_t* plans, const float* const* chi,
                          const float* const* eta, const int* n_lambda, float* const* J,
                          int autotune, rc_batch_t* out);
rc_status rc_batch_run(rc_batch_t batch, void* stream);
rc_status rc_batch_info(rc_batch_t batch, int* launches_per_run, int* lambda_block,
                        int* lambda_per_lane);
/* Number of bound domains that keep their own launch sequence (-1 if batch is NULL). */
int rc_batch_solo_domains(rc_batch_t batch);
void rc_batch_destroy(rc_batch_t batch);

/* One-shot batched solve: rc_batch_create + rc_batch_run + synchronise + rc_batch_destroy. */
rc_status rc_formal_solve_batched(int n, const rc_plan_t* plans, const float* const* chi,
                                  const float* const* eta, const int* n_lambda, float* const* J,
                                  void* stream);

/*
 * rc_formal_solve_mali -- the formal solution with the two extra cascade-0 outputs the
 * MALI population update needs (Sec. 3.3, Eq. 17-19), computed without cancellation:
 *   J_eff  device FP32 [n_lambda][nz][nx] or NULL: J - Lambda* S_local, the mean intensity
 *          without the emission of the cell's own centre-to-edge segment (the effective
 *          intensity I_dagger - Psi* eta_dagger of Eq. 19 with a diagonal operator).  It is
 *          accumulated without that term rather than by subtraction, so it keeps FP32
 *          relative precision in optically thick cells where J ~ S.
 *   alo_c  device FP32 or NULL: 1 - Lambda* = (1/W_0) sum_k exp(-chi d_k), the escape
 *          probability of the cell's own segment (accurate where Lambda* -> 1).
 * J and alo as rc_formal_solve (alo may be NULL).  Requires interval0 >= the centre-to-edge
 * path of every cascade-0 direction (0.5/max(|cos|,|sin|) voxels, e.g. 0.71 for W_0 = 4).
 * Errors: as rc_formal_solve, plus RC_ERR_ARG if interval0 is too short for J_eff.
 */
rc_status rc_formal_solve_mali(rc_plan_t plan, const float* chi, const float* eta, int n_lambda,
                               float* J, float* alo, float* J_eff, float* alo_c, void* stream);

/* ---------------------------------------------------------------------------------------
 * Non-LTE population update (Sec. 3.3): model atom, LTE start, opacity/emissivity from
 * populations, statistical equilibrium with MALI rates, and the iteration driver.
 * Populations and thermodynamic inputs are FP64 (populations span many decades); the
 * formal solution in between is FP32.
 * ------------------------------------------------------------------------------------- */

/* Atom with non-overlapping Gaussian lines in complete redistribution.  Host pointers,
 * copied by rc_atom_create. */
typedef struct {
    int n_levels;          /* 2..8 */
    const double* E_eV;    /* level energies in eV (n_levels), ascending from the ground level */
    const double* g;       /* statistical weights (n_levels) */
    int n_lines;           /* 1..16 */
    const int* lower;      /* lower level of each line */
    const int* upper;      /* upper level of each line (> lower) */
    const double* A_ul;    /* Einstein A of each line, s^-1 */
    int n_per_line;        /* frequencies per line, 2..64 */
    double x_max;          /* grid half-width in Doppler widths at T_ref (uniform in frequency) */
    double T_ref;          /* K */
    double mass_amu;       /* atomic mass */
} rc_atom_desc;

typedef struct rc_atom_s* rc_atom_t;

/* Derives the line constants (nu0, B_ul = A c^2/(2 h nu0^3), B_lu = g_u/g_l B_ul, f_lu, the
 * frequency grid and trapezoid weights) and uploads them to the current device.
 * Errors: RC_ERR_ARG, RC_ERR_OOM, RC_ERR_CUDA. */
rc_status rc_atom_create(const rc_atom_desc* desc, rc_atom_t* out);
void rc_atom_destroy(rc_atom_t atom);
/* Number of line wavelengths (n_lines * n_per_line); the wavelength index is
 * line * n_per_line + k. */
int rc_atom_n_lambda(rc_atom_t atom);

/*
 * rc_lte -- LTE start (Sec. 3.3): pure-hydrogen Saha ionisation at (T, n_H) gives n_e and
 * the neutral density n_atom; the levels follow Boltzmann over the model's levels.
 * Device FP64 arrays of ncell cells; pops is [n_levels][ncell].  Asynchronous.
 * Errors: RC_ERR_ARG, RC_ERR_CUDA.
 */
rc_status rc_lte(rc_atom_t atom, const double* T, const double* nH, long long ncell, double* ne,
                 double* n_atom, double* pops, void* stream);

/*
 * rc_emis_opac -- line opacity and emissivity at every grid frequency (the inputs of the RTE,
 * Sec. 3.2): chi = (h nu0/4 pi)(n_l B_lu - n_u B_ul) phi, eta = (h nu0/4 pi) n_u A_ul phi,
 * phi the Gaussian profile at the local Doppler width renormalised so that sum_k w_k phi_k = 1.
 * T, pops device FP64; chi [m^-1] and eta [W m^-3 Hz^-1 sr^-1] device FP32
 * [n_lambda][ncell].  Asynchronous.  Errors: RC_ERR_ARG, RC_ERR_CUDA.
 */
rc_status rc_emis_opac(rc_atom_t atom, const double* T, const double* pops, long long ncell,
                       float* chi, float* eta, void* stream);

/*
 * rc_stat_eq -- statistical equilibrium Gamma n = 0 per cell (Sec. 3.3, Eq. 20) with the
 * same-preconditioning MALI rates of a diagonal operator (Eq. 18-19):
 *   R_lu = B_lu Jeff_bar,  R_ul = A_ul (1 - Lambda*)_bar + B_ul Jeff_bar,
 * bars = sum_k w_k phi_k (.), plus van Regemorter collisions (C_ul from detailed balance).
 * Only off-diagonal rates are accumulated; the diagonal is minus the column sum; the row of
 * the most populated level is replaced by sum n = n_atom; the system is solved in FP64.
 *   J_eff, alo_c   device FP32 [n_lambda][ncell] from rc_formal_solve_mali.  alo_c = NULL
 *                  means Lambda* = 0 (plain Lambda iteration; pass J as J_eff).
 *   pops           device FP64 [n_levels][ncell], in: previous iterate, out: new populations.
 *   max_rel_change host FP64 out (may be NULL): max over cells and levels of
 *                  |n_new - n_old| / n_new.  If non-NULL the call synchronises the stream.
 * Errors: RC_ERR_ARG, RC_ERR_CUDA.
 */
rc_status rc_stat_eq(rc_atom_t atom, const double* T, const double* ne, const double* n_atom,
                     const float* J_eff, const float* alo_c, long long ncell, double* pops,
                     double* max_rel_change, void* stream);

/*
 * rc_stat_eq in two halves, for a non-LTE iteration whose wavelengths are split between
 * processes (each runs the formal solution of its own range; Sec. 3.6 treats wavelengths as
 * independent within an iteration).  The rates of Sec. 3.3 depend on the radiation field only
 * through two integrals per line and cell, Jeff_bar = sum_k w_k phi_k J_eff and
 * (1 - Lambda*)_bar = sum_k w_k phi_k (1 - Lambda*), and an integral over a range of a line's
 * wavelengths is a partial sum of it (the profile is normalised over the whole line).
 * rc_line_integrals -- the integrals over the atom's grid wavelengths
 *   [lambda_begin, lambda_begin + lambda_count) (global indices, line after line):
 *   J_eff, alo_c   device FP32 [lambda_count][ncell], the range's wavelengths only; alo_c NULL
 *                  means Lambda* = 0.
 *   out            device FP64 [n_lines][2][ncell]: (Jeff_bar, (1 - Lambda*)_bar) of each line
 *                  over the range (0 for lines outside it).  Asynchronous.
 * rc_stat_eq_integrals -- the update of rc_stat_eq from integrals summed over every range (an
 *   all-reduce of the n_lines x 2 x ncell FP64 partials: 6 per cell for the 3-level atom);
 *   T, ne, n_atom, pops, max_rel_change as rc_stat_eq.  Every process holding the same sums
 *   computes the same populations.  With one range covering all wavelengths the two calls
 *   equal rc_stat_eq bit for bit.
 * Errors: RC_ERR_ARG (NULL arguments, range outside the grid), RC_ERR_CUDA.
 */
rc_status rc_line_integrals(rc_atom_t atom, const double* T, const float* J_eff, const float* alo_c,
                            int lambda_begin, int lambda_count, long long ncell, double* out,
                            void* stream);
rc_status rc_stat_eq_integrals(rc_atom_t atom, const double* T, const double* ne,
                               const double* n_atom, const double* integrals, long long ncell,
                               double* pops, double* max_rel_change, void* stream);

/*
 * rc_nlte_solve -- the non-LTE iteration (Sec. 3.3): repeat {rc_emis_opac, rc_formal_solve_mali,
 * rc_stat_eq} from the populations in `pops` until the maximum relative change drops below
 * tol (Sec. 4.2 uses 1e-3) or max_iter iterations ran.  The plan's grid must have
 * nx * nz = ncell cells and its voxel_size in metres.  history (host, max_iter entries, may be
 * NULL) receives the change of every iteration.  Synchronises once per iteration (one 8-byte
 * copy).  Returns RC_OK on convergence, RC_ERR_NOT_CONVERGED after max_iter iterations
 * (pops then holds the last iterate).
 */
rc_status rc_nlte_solve(rc_plan_t plan, rc_atom_t atom, const double* T, const double* ne,
                        const double* n_atom, double* pops, double tol, int max_iter,
                        int* iterations, double* final_change, double* history, void* stream);

/* ---------------------------------------------------------------------------------------
 * Surrogate seed of the non-LTE iteration.  The paper has no learned component; this is a
 * start for the iteration of Sec. 3.3 in place of LTE, and LTE stays the fallback.
 * Network: x (6 features) -> tanh(W1 xn + b1) (64) -> tanh(W2 h1 + b2) (64) -> W3 h2 + b3 (3),
 * xn the standardised input; parameters flattened as W1[64][6], b1, W2[64][64], b2, W3[3][64],
 * b3 (4803 floats).  FP32 master weights and Adam moments; the passes multiply with the
 * bfloat16-rounded weights and accumulate in FP32.
 * Features of a cell: log10 T, log10 n_e, log10 n_H and log10 J at the centre wavelength of
 * each of the first three lines from the first (LTE) formal solution.  Targets: log10 of the
 * departure coefficients n_i / n_i(LTE) of the three levels.
 * ------------------------------------------------------------------------------------- */
typedef struct rc_mlp_s* rc_mlp_t;
/* Glorot-uniform weights from `seed`, zero biases, identity standardisation. */
rc_status rc_mlp_create(unsigned long long seed, rc_mlp_t* out);
void rc_mlp_destroy(rc_mlp_t net);
int rc_mlp_n_params(rc_mlp_t net);
/* Host copies of the parameters and the standardisation (mean, std of each feature); any
 * pointer may be NULL.  Setting parameters resets the Adam state.  Synchronous. */
rc_status rc_mlp_set_params(rc_mlp_t net, const float* theta, const float* mean, const float* std_);
rc_status rc_mlp_get_params(rc_mlp_t net, float* theta, float* mean, float* std_);
/* Standardisation from the mean and standard deviation of device features X [N][6]. */
rc_status rc_mlp_fit_normalization(rc_mlp_t net, const float* X, long long N, void* stream);
/* Y [B][3] = network(X [B][6]); device buffers, asynchronous. */
rc_status rc_mlp_forward(rc_mlp_t net, const float* X, long long B, float* Y, void* stream);
/* Tensor cores for the network (enable is a bit set; 0, the default, uses FP32 FMAs with the
 * bf16 weights everywhere):
 *   RC_MLP_TC_INFERENCE (1)  rc_mlp_forward (and so rc_surrogate_seed) runs the 64 x 64 layer on
 *                            the tensor cores (tcgen05.mma, bf16 h1 and W2 from shared memory,
 *                            FP32 accumulator in tensor memory, 128 samples per CTA);
 *   RC_MLP_TC_TRAINING (2)   rc_mlp_loss_grad and rc_mlp_train run the three 64-wide products of
 *                            a tile (h1 W2^T, dh2 W2, dh2^T h1) on the tensor cores, each FP32
 *                            activation passed as two bf16 parts (hi + lo, ~16 significant bits),
 *                            so the gradient keeps the FMA path's accuracy; per-tile partial
 *                            gradients are summed in a fixed order as on the FMA path
 *                            (reproducible bit for bit, though not bit-equal to the FMA path).
 * rc_mlp_tensor_core_status reports RC_ERR_TIMEOUT if a tensor-core wait ever ran out (the
 * kernel then skipped its outputs).  A CTA whose wait ran out waits once more, 8x as long,
 * before it releases its tensor memory; if the MMAs still have not completed it leaves the
 * 64 columns allocated rather than free memory a late MMA could still write, and the message
 * says so (later tensor-core launches on that SM have less tensor memory; recreate the
 * context).  A training tile whose wait ran out stores a zero gradient. */
enum { RC_MLP_TC_INFERENCE = 1, RC_MLP_TC_TRAINING = 2 };
rc_status rc_mlp_use_tensor_cores(rc_mlp_t net, int enable);
rc_status rc_mlp_tensor_core_status(rc_mlp_t net);

/* Self-test of the library's bounded device-side wait (no counterpart in the paper): one CTA
 * waits on an mbarrier that nobody completes, through the same bounded poll the tensor-core
 * kernel uses, gives up after ~0.3 ms and reports it.  Returns RC_ERR_TIMEOUT when the wait
 * gave up as designed (the expected result; the CUDA context stays usable), RC_ERR_CUDA on a
 * launch/copy failure or if the wait did not give up.  Synchronous on `stream`. */
rc_status rc_selftest_bounded_wait(void* stream);
/* Mean-squared-error loss over B samples and its gradient (device outputs, either may be NULL). */
rc_status rc_mlp_loss_grad(rc_mlp_t net, const float* X, const float* Y_target, long long B,
                           float* grad, float* loss, void* stream);
/* `steps` Adam steps (beta 0.9/0.999, eps 1e-8) on minibatches of `batch` rows drawn from
 * device X [N][6], Y_target [N][3] by a counter-based generator (splitmix64 of the network's
 * seed and step).  loss_history (host, `steps` entries, may be NULL: then no synchronisation)
 * receives each minibatch loss. */
rc_status rc_mlp_train(rc_mlp_t net, const float* X, const float* Y_target, long long N, int batch,
                       int steps, float lr, float* loss_history, void* stream);
/* The surrogate's life cycle under the names of the method's interface (no counterpart in the
 * paper): rc_surrogate_init = rc_mlp_create; rc_surrogate_train_step = one Adam step of
 * rc_mlp_train (loss: host float or NULL; NULL does not synchronise); rc_surrogate_predict =
 * rc_mlp_forward (log10 departure coefficients [B][3] from features [B][6]). */
rc_status rc_surrogate_init(unsigned long long seed, rc_mlp_t* out);
rc_status rc_surrogate_train_step(rc_mlp_t net, const float* X, const float* Y_target, long long N,
                                  int batch, float lr, float* loss, void* stream);
rc_status rc_surrogate_predict(rc_mlp_t net, const float* X, long long B, float* Y, void* stream);
/* Features X [ncell][6] from device T, n_e, n_H (FP64) and J [n_lambda][ncell] (FP32). */
rc_status rc_surrogate_features(rc_atom_t atom, const double* T, const double* ne, const double* nH,
                                const float* J, long long ncell, float* X, void* stream);
/* Targets Y [ncell][3] = log10(n_i / n_i(LTE)) from device populations (3-level atoms). */
rc_status rc_surrogate_targets(rc_atom_t atom, const double* T, const double* n_atom,
                               const double* pops, long long ncell, float* Y, void* stream);
/* Seeded populations: n_i = 10^y_i n_i(LTE) renormalised to n_atom, y = network(X); cells whose
 * output is not finite and positive fall back to LTE (their count -> *n_fallback, host, may be
 * NULL: then asynchronous).  Allocates a forward scratch on the network on first use. */
rc_status rc_surrogate_seed(rc_atom_t atom, rc_mlp_t net, const float* X, const double* T,
                            const double* n_atom, long long ncell, double* pops, int* n_fallback,
                            void* stream);

/*
 * rc_emergent -- emergent intensity by single-pass front-to-back long characteristics
 * (Sec. 3.9): each ray starts at its origin and accumulates, outward along its direction,
 * exp(-tau_before) S (1 - exp(-chi ds)) of every voxel piece it crosses to the domain edge --
 * the intensity reaching the origin from that direction -- for every wavelength.
 *   rays     device FP32 [n_rays][4], 16-byte aligned: origin (x, z) in voxels, unit
 *            direction (wx, wz).  Origins may lie outside the domain.
 *   mu       inclination to the invariant axis, 0 <= mu < 1: the path per projected length is
 *            1/sqrt(1 - mu^2) (2D invariance, Sec. 3.1).
 *   I        device FP32 [n_lambda][n_rays], written.
 *   contrib  device FP32 [n_lambda][nz][nx] or NULL: each piece's contribution added to its
 *            cell (the contribution function summed over the rays); the caller zeroes it.
 * Uses the plan's grid, voxel size, packing scratch and (if set) active cells.  Asynchronous.
 * Errors: RC_ERR_ARG, RC_ERR_OOM, RC_ERR_CUDA.
 */
rc_status rc_emergent(rc_plan_t plan, const float* chi, const float* eta, int n_lambda,
                      const float* rays, long long n_rays, float mu, float* I, float* contrib,
                      void* stream);

/* One-line message for the calling thread's last error ("" if none). */
const char* rc_last_error(void);

/* Static name of a status code. */
const char* rc_status_string(rc_status s);

#ifdef __cplusplus
}
#endif

#endif /* RCX_H */
