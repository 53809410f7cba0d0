// rcx_fs_kernels.cu -- sm_103a kernels of the radiance-cascade formal solution.
//
// Work decomposition (one launch per cascade, top cascade first):
//   * The opacity/emissivity slabs are first packed into a wavelength-blocked
//     layout [lambda block][cell][LB] of (chi' = chi voxel log2 e, S = eta/chi)
//     pairs.  One ray is marched for the LB wavelengths of a block by LB/VL lanes,
//     each carrying VL wavelengths; the lanes of a ray read one contiguous
//     8*LB-byte run per voxel, and every DDA instruction of a lane serves VL
//     crossings.  A warp holds the rays of 32*VL/LB neighbouring directions of one
//     probe, which walk the grid in near lock-step.
//   * Each lane marches front to back (Sec. 3.2 allows either order) with the
//     piecewise-constant update of Eq. 16 in FP32, keeping the running
//     transmittance T:  I += T S (1 - e^{-dtau}),  T *= e^{-dtau}.
//   * The merge of Sec. 2.3.1 is fused into the same kernel: the lane reads, on each
//     of the four bracketing upper probes, the average of the four child rays of its
//     direction (stored once by the upper cascade, one vector per probe), interpolates
//     bilinearly with the edge clamp of Sec. 2.5 and forms R = I + T * upper (Eq. 11,
//     the nearer interval attenuating the farther one).  The four sibling rays of a
//     probe then sum their R across lane groups and store the average for the cascade
//     below.
//   * Long cascades over fields larger than L2 run strip by strip (level_split_kernel).
//   * Cascade 0 folds the W_0 directions of its probe (a cell centre) into J
//     (Eq. 1) and, optionally, the diagonal operator of Eq. 17.
// No tensor cores: the march is a gather walk, not a contraction.
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rcx_internal.h"

// Resident CTAs per SM the cascade kernels are compiled for (register budget
// 65536 / (32 x kWarpsPerCta threads x this)), set for 48 warps per SM.  48 warps (40
// registers) measured 7% faster than 40 (48 registers) on the 1024^2 x 64 x 8-cascade
// workload: the extra resident warps hide more of the gather latency.
#ifndef RCX_MIN_CTAS
#define RCX_MIN_CTAS (48 / RCX_WARPS_PER_CTA)
#endif
// With 8 wavelengths per lane the field data in flight alone takes 16 registers: a 40-register
// budget spills inside the march loop, so those instantiations get a budget of their own
// (32 warps/SM: 676 slices/s at 1024^2 x 64, 565 at 40 warps with spills, 803 with 4 per lane).
#ifndef RCX_MIN_CTAS_VL8
#define RCX_MIN_CTAS_VL8 (32 / RCX_WARPS_PER_CTA)
#endif
// Cascade 0 for J alone (no operator outputs, dense): 32 warps/SM measured 0.98 ms per 1024^2
// 64-wavelength step against 1.03 ms at 24.
#ifndef RCX_MIN_CTAS_L0J
#define RCX_MIN_CTAS_L0J (32 / RCX_WARPS_PER_CTA)
#endif
#ifndef RCX_MIN_CTAS_L0
#define RCX_MIN_CTAS_L0 (24 / RCX_WARPS_PER_CTA)
#endif

namespace rcx {

template <int VL>
constexpr int min_ctas() { return VL >= 8 ? RCX_MIN_CTAS_VL8 : RCX_MIN_CTAS; }
// The strip kernel in CTAs of WPC warps, at the same warps per SM (same registers).  Strips
// of 4 and more per cascade run in 8-warp CTAs: at 2048^2 (8 strips) cascade 5 took 349.7 ms
// per 64-wavelength step with 8-warp CTAs against 386.8 with 4; at 1024^2 (2 strips) 4-warp
// CTAs are faster (32.8 against 33.5 ms).
constexpr int kSplitWideWarps = 8, kSplitWideFrom = 4;   // warps per CTA, from this many strips
template <int VL, int WPC>
constexpr int min_ctas_w() { return (VL >= 8 ? 32 : 48) / WPC; }

// ---------------------------------------------------------------------------
// storage of merged intervals: FP32, or FP16/BF16 with a per-block scale
// ---------------------------------------------------------------------------
template <typename TS>
struct Store;

template <>
struct Store<float> {
    static __device__ __forceinline__ void store(float* p, float v) { *p = v; }
};

template <>
struct Store<__half> {
    static __device__ __forceinline__ void store(__half* p, float v) { *p = __float2half_rn(v); }
};

template <>
struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float v) {
        *p = __float2bfloat16_rn(v);
    }
};

// VL consecutive stored values (VL * sizeof(TS)-aligned) as floats, and back.
template <typename TS, int VL>
__device__ __forceinline__ void load_vec(const TS* __restrict__ p, float (&v)[VL]) {
    if constexpr (std::is_same<TS, float>::value) {
        if constexpr (VL == 1) {
            v[0] = __ldg(p);
        } else if constexpr (VL == 2) {
            const float2 a = __ldg(reinterpret_cast<const float2*>(p));
            v[0] = a.x;
            v[1] = a.y;
        } else {
#pragma unroll
            for (int j = 0; j < VL; j += 4) {
                const float4 a = __ldg(reinterpret_cast<const float4*>(p + j));
                v[j] = a.x;
                v[j + 1] = a.y;
                v[j + 2] = a.z;
                v[j + 3] = a.w;
            }
        }
    } else {
        using T2 = typename std::conditional<std::is_same<TS, __half>::value, __half2,
                                             __nv_bfloat162>::type;
        if constexpr (VL == 1) {
            v[0] = (float)p[0];
        } else {
            // VL / 2 pairs in one load of VL * 2 bytes
            T2 h[VL / 2];
            if constexpr (VL == 2) *reinterpret_cast<unsigned*>(h) = __ldg(reinterpret_cast<const unsigned*>(p));
            if constexpr (VL == 4) *reinterpret_cast<uint2*>(h) = __ldg(reinterpret_cast<const uint2*>(p));
            if constexpr (VL == 8) *reinterpret_cast<uint4*>(h) = __ldg(reinterpret_cast<const uint4*>(p));
#pragma unroll
            for (int j = 0; j < VL / 2; ++j) {
                const float2 f = std::is_same<TS, __half>::value
                                     ? __half22float2(*reinterpret_cast<__half2*>(&h[j]))
                                     : __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&h[j]));
                v[2 * j] = f.x;
                v[2 * j + 1] = f.y;
            }
        }
    }
}

template <typename TS, int VL>
__device__ __forceinline__ void store_vec(TS* __restrict__ p, const float (&v)[VL]) {
    if constexpr (std::is_same<TS, float>::value) {
        if constexpr (VL == 1) {
            p[0] = v[0];
        } else if constexpr (VL == 2) {
            *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
        } else {
#pragma unroll
            for (int j = 0; j < VL; j += 4)
                *reinterpret_cast<float4*>(p + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
    } else if constexpr (VL == 1) {
        Store<TS>::store(p, v[0]);
    } else {
        // VL / 2 pairs, each rounded to nearest like Store, written in one store of VL * 2 bytes
        unsigned h[VL / 2];
#pragma unroll
        for (int j = 0; j < VL / 2; ++j) {
            if constexpr (std::is_same<TS, __half>::value) {
                const __half2 t = __floats2half2_rn(v[2 * j], v[2 * j + 1]);
                h[j] = *reinterpret_cast<const unsigned*>(&t);
            } else {
                const __nv_bfloat162 t = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                h[j] = *reinterpret_cast<const unsigned*>(&t);
            }
        }
        if constexpr (VL == 2) *reinterpret_cast<unsigned*>(p) = h[0];
        if constexpr (VL == 4) *reinterpret_cast<uint2*>(p) = make_uint2(h[0], h[1]);
        if constexpr (VL == 8) *reinterpret_cast<uint4*>(p) = make_uint4(h[0], h[1], h[2], h[3]);
    }
}

// ---------------------------------------------------------------------------
// one radiance interval
// ---------------------------------------------------------------------------

// The packed opacity is chi per voxel times log2(e), so exp(-chi ds) = 2^(-y) with
// y = chi' ds: one multiply and one MUFU.EX2 per crossing.
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.69314718055994531f;

__device__ __forceinline__ float exp2_neg(float y) {
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-y));
    return e;
}

// 1 - 2^(-y) for y >= 0 without cancellation: the Taylor series of 1 - e^(-x),
// x = y ln 2, to second order below y = 2^-7 (truncation below x^2/6 ~ 5e-6
// relative), 1 - e otherwise (e = 2^(-y) already computed).  ex2.approx measured
// within 2.1 ulp on B300, so 1 - e is within 2e-5 relative for y >= 2^-7.
__device__ __forceinline__ float one_minus_exp2_neg(float y, float e) {
    constexpr float a1 = kLn2;
    constexpr float a2 = -0.5f * kLn2 * kLn2;
    const float s = y * fmaf(y, a2, a1);
    return y < 0.0078125f ? s : 1.0f - e;
}

// VL consecutive (chi', S) pairs of one voxel for this lane's wavelengths.
template <int VL>
struct Voxel {
    float2 v[VL];
    __device__ __forceinline__ void load(const float2* __restrict__ p) {
        if constexpr (VL == 1) {
            v[0] = __ldg(p);
        } else if constexpr (VL % 4 == 0) {
            // 32-byte loads (the lane's offset is a multiple of 4 pairs, the field 128 B
            // aligned): one load instruction per 4 wavelengths
#pragma unroll
            for (int j = 0; j < VL; j += 4)
                asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=f"(v[j].x), "=f"(v[j].y), "=f"(v[j + 1].x), "=f"(v[j + 1].y),
                               "=f"(v[j + 2].x), "=f"(v[j + 2].y), "=f"(v[j + 3].x), "=f"(v[j + 3].y)
                             : "l"(p + j));
        } else {
#pragma unroll
            for (int j = 0; j < VL; j += 2) {
                const float4 q = __ldg(reinterpret_cast<const float4*>(p) + j / 2);
                v[j] = make_float2(q.x, q.y);
                v[j + 1] = make_float2(q.z, q.w);
            }
        }
    }
};

// R_{a,b}(o, w) for the VL wavelengths of this lane.  Front-to-back DDA over the
// uniform grid (Sec. 3.2 allows either order).  The parameter of the k-th x face
// after entry is tx0 + k dtx (one FMA, no accumulated error), and the domain exit
// is evaluated with the same expression, so the walk ends exactly on it and never
// leaves the grid.  The advance is predicated (no divergent branch between rays
// of a warp that step along different axes), and the voxel address is a running
// 32-bit offset (cell * LB + lane_off).
// With SPLIT_FIRST the emission of the first piece (for a cascade-0 ray: the probe's
// own cell from its centre to its edge) goes to I0 instead of I.  With CONTRIB every
// piece's contribution T S (1 - e^{-dtau}) is also added to contrib[j * ncell + cell] for the
// lane's first n_valid wavelengths (the contribution function of Sec. 3.9).  Returns false
// when the interval misses the box (I = 0, T = 1).
template <int LB, int VL, bool SPLIT_FIRST = false, bool CONTRIB = false>
__device__ __forceinline__ bool march_interval(const float2* __restrict__ F, int nx, int nz,
                                               int x0, int x1,
                                               float ox, float oz, float wx, float wz,
                                               float a, float b, int lane_off, int max_steps,
                                               float (&I)[VL], float (&T)[VL], float (&I0)[VL],
                                               float* contrib = nullptr, int n_valid = 0,
                                               long long ncell = 0) {
#pragma unroll
    for (int j = 0; j < VL; ++j) {
        I[j] = 0.0f;
        T[j] = 1.0f;
        I0[j] = 0.0f;
    }
    const float invx = wx != 0.0f ? 1.0f / wx : 1e30f;
    const float invz = wz != 0.0f ? 1.0f / wz : 1e30f;
    // entry into the box [x0, x1] x [0, nz] (the domain, or a strip of it; free space
    // outside the domain, Sec. 3.4); nx is the row stride of the field
    const float tx0 = ((float)x0 - ox) * invx, tx1 = ((float)x1 - ox) * invx;
    const float tz0 = (0.0f - oz) * invz, tz1 = ((float)nz - oz) * invz;
    const float tlo = fmaxf(a, fmaxf(fminf(tx0, tx1), fminf(tz0, tz1)));
    if (!(tlo < fminf(b, fminf(fmaxf(tx0, tx1), fmaxf(tz0, tz1))))) return false;

    const bool upx = wx > 0.0f, upz = wz > 0.0f;
    const float ex = ox + tlo * wx, ez = oz + tlo * wz;
    int ix = (int)floorf(ex), iz = (int)floorf(ez);
    if (!upx && (float)ix == ex) --ix;   // entering through a face while moving down
    if (!upz && (float)iz == ez) --iz;
    ix = min(max(ix, x0), x1 - 1);
    iz = min(max(iz, 0), nz - 1);

    // face parameters: first face after entry and spacing between faces (+inf along an axis
    // the ray does not move on: it never crosses those faces, and their exit term never binds)
    const float fx0 = (float)(upx ? ix + 1 : ix), fz0 = (float)(upz ? iz + 1 : iz);
    const float tfx = wx != 0.0f ? (fx0 - ox) * invx : INFINITY;
    const float tfz = wz != 0.0f ? (fz0 - oz) * invz : INFINITY;
    const float dtx = fabsf(invx), dtz = fabsf(invz);
    // exit: last face inside the domain, with the same expression as the walk
    const float kx_end = (float)(upx ? x1 - 1 - ix : ix - x0);
    const float kz_end = (float)(upz ? nz - 1 - iz : iz);
    const float thi = fminf(b, fminf(fmaf(kx_end, dtx, tfx), fmaf(kz_end, dtz, tfz)));

    float kx = 0.0f, kz = 0.0f;
    float tnx = tfx, tnz = tfz;
    int off = (iz * nx + ix) * LB + lane_off;
    const int dox = upx ? LB : -LB;
    const int doz = upz ? nx * LB : -nx * LB;
    float t = tlo;
    // The walk does not depend on the field, so the next voxel is fetched one step
    // ahead: two loads per lane are in flight while the current voxel is integrated.
    // After the last step that fetch is one voxel past the exit face (up to a row outside
    // the block); the packed field is allocated with a guard band of a row of voxels on
    // both sides, so it reads allocated memory, and the value is never used.
    if constexpr (VL == 8 && !SPLIT_FIRST && !CONTRIB) {
        // Eight wavelengths per lane in two halves of four: the next voxel's first half is
        // fetched as soon as this voxel's first half has been integrated, and its second half
        // after the second, so each half is prefetched about half a step ahead and only 16
        // registers of field data are live (instead of 32 for a whole voxel ahead).
        Voxel<4> lo, hi;
        lo.load(F + off);
        hi.load(F + off + 4);
        for (int step = 0; step < max_steps; ++step) {
            const bool stepx = tnx <= tnz;
            const float tn = fminf(fminf(tnx, tnz), thi);
            const float ds = tn - t;
            const int off_next = off + (stepx ? dox : doz);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float y = lo.v[j].x * ds;
                const float e = exp2_neg(y);
                const float om = one_minus_exp2_neg(y, e);
                I[j] = fmaf(T[j] * lo.v[j].y, om, I[j]);
                T[j] *= e;
            }
            lo.load(F + off_next);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float y = hi.v[j].x * ds;
                const float e = exp2_neg(y);
                const float om = one_minus_exp2_neg(y, e);
                I[4 + j] = fmaf(T[4 + j] * hi.v[j].y, om, I[4 + j]);
                T[4 + j] *= e;
            }
            hi.load(F + off_next + 4);
            if (tn >= thi) break;
            if (stepx) {
                kx += 1.0f;
                tnx = fmaf(kx, dtx, tfx);
            } else {
                kz += 1.0f;
                tnz = fmaf(kz, dtz, tfz);
            }
            off = off_next;
            t = tn;
        }
        return true;
    }
    Voxel<VL> cur;
    cur.load(F + off);
    for (int step = 0; step < max_steps; ++step) {
        const bool stepx = tnx <= tnz;
        const float tn = fminf(fminf(tnx, tnz), thi);
        const float ds = tn - t;
        const int off_next = off + (stepx ? dox : doz);
        Voxel<VL> nxt;
        nxt.load(F + off_next);
#pragma unroll
        for (int j = 0; j < VL; ++j) {
            const float y = cur.v[j].x * ds;
            const float e = exp2_neg(y);
            const float om = one_minus_exp2_neg(y, e);
            if (SPLIT_FIRST && step == 0)
                I0[j] = cur.v[j].y * om;
            else
                I[j] = fmaf(T[j] * cur.v[j].y, om, I[j]);
            if (CONTRIB && j < n_valid)
                atomicAdd(contrib + (size_t)j * ncell + (off - lane_off) / LB,
                          T[j] * cur.v[j].y * om);
            T[j] *= e;
        }
        if (tn >= thi) break;
        if (stepx) {
            kx += 1.0f;
            tnx = fmaf(kx, dtx, tfx);
        } else {
            kz += 1.0f;
            tnz = fmaf(kz, dtz, tfz);
        }
        off = off_next;
        cur = nxt;
        t = tn;
    }
    return true;
}

// Storage scale of lambda block lb: 16-bit merged intervals are stored divided by a
// per-block scale (the plan always provides the scales with 16-bit storage); FP32 storage
// has none (known at compile time).
template <typename TS>
__device__ __forceinline__ float storage_scale(const LevelArgs& A, int lb) {
    if constexpr (std::is_same<TS, float>::value) return 1.0f;
    else return __ldg(A.scale + lb);
}

// Column and row of a probe (or cell) index on a grid P wide.  Probe and cell counts are
// below 2^31 (rc_plan keeps nx nz LB below it), so the division runs in 32 bits.
__device__ __forceinline__ void grid_xy(long long idx, int P, int& x, int& z) {
    const unsigned u = (unsigned)idx, zz = u / (unsigned)P;
    z = (int)zz;
    x = (int)(u - zz * (unsigned)P);
}

// Clamped bilinear coordinate of a cascade-i probe index m in the index space
// of cascade i+1 (probe positions (m+1/2) 2^i and (j+1/2) 2^(i+1)).
__device__ __forceinline__ void upper_coord(int m, int P_up, int& j0, int& j1, float& f) {
    float u = 0.5f * (float)m - 0.25f;
    u = fminf(fmaxf(u, 0.0f), (float)(P_up - 1));
    j0 = (int)u;
    j1 = min(j0 + 1, P_up - 1);
    f = u - (float)j0;
}

// Merged intervals are stored as child-cone averages: for each probe b of a cascade and
// each direction k of the cascade below, 1/4 sum of the probe's children 4k..4k+3 (Eq. 11
// needs only that average), at [(b W + k) LB + l] with W the lower cascade's direction count.
// Each stored value is read by the 16 lower probes around b, so averaging once at the
// store saves three quarters of the merge's reads.

// Bilinearly weighted child averages of the four bracketing upper probes, for the lane's
// VL wavelengths starting at l.
template <int LB, int VL, typename TS>
__device__ __forceinline__ void upper_radiance(const TS* __restrict__ Rup, long long b00,
                                               long long b01, long long b10, long long b11,
                                               float fx, float fz, int W, int k, int l,
                                               float (&up)[VL]) {
    float c00[VL], c01[VL], c10[VL], c11[VL];
    load_vec<TS, VL>(Rup + (size_t)(b00 * W + k) * LB + l, c00);
    load_vec<TS, VL>(Rup + (size_t)(b01 * W + k) * LB + l, c01);
    load_vec<TS, VL>(Rup + (size_t)(b10 * W + k) * LB + l, c10);
    load_vec<TS, VL>(Rup + (size_t)(b11 * W + k) * LB + l, c11);
#pragma unroll
    for (int j = 0; j < VL; ++j) {
        const float r0 = fmaf(fx, c01[j] - c00[j], c00[j]);
        const float r1 = fmaf(fx, c11[j] - c10[j], c10[j]);
        up[j] = fmaf(fz, r1 - r0, r0);
    }
}

// The bilinear fix (Sec. 2.5) for the ray of probe (px, pz) in direction d starting at
// distance a: the segment from its start A = o + a d to the start of the child interval of
// each bracketing upper probe, B = x_b + a_up d, is marched, merged with that probe's child
// average, and the four results are weighted bilinearly.  R[j] receives the sum.
template <int LB, int VL, typename TS>
__device__ __forceinline__ void fixed_rays(const LevelArgs& A, const float2* __restrict__ F,
                                           const TS* __restrict__ Rup, float sc, int px, int pz,
                                           float ox, float oz, float2 d, int k, int lane_off,
                                           float (&R)[VL]) {
    int jx[2], jz[2];
    float fx, fz;
    upper_coord(px, A.Px_up, jx[0], jx[1], fx);
    upper_coord(pz, A.Pz_up, jz[0], jz[1], fz);
    const float sp_up = 2.0f * A.spacing;
    const float Ax = ox + A.a * d.x, Az = oz + A.a * d.y;
#pragma unroll
    for (int j = 0; j < VL; ++j) R[j] = 0.0f;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float w = (r ? fx : 1.0f - fx) * (q ? fz : 1.0f - fz);
            if (w == 0.0f) continue;
            const float dx = ((float)jx[r] + 0.5f) * sp_up + A.a_up * d.x - Ax;
            const float dz = ((float)jz[q] + 0.5f) * sp_up + A.a_up * d.y - Az;
            const float L = sqrtf(dx * dx + dz * dz);
            float I[VL], T[VL], I0[VL];
            if (L > 0.0f) {
                const float iL = 1.0f / L;
                march_interval<LB, VL>(F, A.nx, A.nz, 0, A.nx, Ax, Az, dx * iL, dz * iL, 0.0f, L,
                                       lane_off, A.max_steps, I, T, I0);
            } else {
#pragma unroll
                for (int j = 0; j < VL; ++j) {
                    I[j] = 0.0f;
                    T[j] = 1.0f;
                }
            }
            const long long b = (long long)jz[q] * A.Px_up + jx[r];
            float up[VL];
            load_vec<TS, VL>(Rup + (size_t)(b * A.W + k) * LB + lane_off, up);
#pragma unroll
            for (int j = 0; j < VL; ++j) R[j] = fmaf(w, fmaf(T[j], up[j] * sc, I[j]), R[j]);
        }
}

struct Bilinear {
    long long b00, b01, b10, b11;
    float fx, fz;
    __device__ __forceinline__ Bilinear(int px, int pz, int Px_up, int Pz_up) {
        int jx0, jx1, jz0, jz1;
        upper_coord(px, Px_up, jx0, jx1, fx);
        upper_coord(pz, Pz_up, jz0, jz1, fz);
        b00 = (long long)jz0 * Px_up + jx0;
        b01 = (long long)jz0 * Px_up + jx1;
        b10 = (long long)jz1 * Px_up + jx0;
        b11 = (long long)jz1 * Px_up + jx1;
    }
};

// ---------------------------------------------------------------------------
// cascades >= 1: march + merge, store the merged interval
// ---------------------------------------------------------------------------
template <int LB, int VL, typename TS>
__device__ __forceinline__ void store_child_average(const LevelArgs& A, int lb, bool valid,
                                                    long long sray, int lane_off, float (&R)[VL]);

// One CTA-sized chunk `cta` of the rays of lambda block `lb` of one cascade.  The four
// rays 4m..4m+3 of a probe (consecutive directions: the children of direction m of the
// cascade below) are summed across their lane groups and stored once as their average.
// FAST: the direction count is a power of two and every probe is marched (no sparse list),
// both known at compile time.
template <int LB, int VL, typename TS, bool HAS_UP, bool FIX = false, bool FAST = false>
__device__ __forceinline__ void level_body(const LevelArgs& A, int lb, long long cta) {
    constexpr int LPR = LB / VL;   // lanes per ray
    constexpr int G = 32 / LPR;    // rays per warp
    const int lane = threadIdx.x & 31;
    const int g = lane / LPR, q = lane % LPR;
    const long long wid = cta * kWarpsPerCta + (threadIdx.x >> 5);
    const long long ray = wid * G + g;
    const int lane_off = q * VL;
    // ray counts of cascades >= 1 are multiples of 4, so a group of four is valid or not as a
    // whole; invalid lanes still take part in the group sum below
    const bool valid = ray < A.rays;

    float R[VL];
    long long sray = 0;            // the ray's slot in the merged storage
#pragma unroll
    for (int j = 0; j < VL; ++j) R[j] = 0.0f;
    if (valid) {
        int k;
        long long probe;
        if (FAST || A.Wshift >= 0) {
            k = (int)(ray & (A.W - 1));
            probe = ray >> A.Wshift;
        } else {
            k = (int)(ray % A.W);
            probe = ray / A.W;
        }
        if (!FAST && A.probe_list) probe = A.probe_list[probe];   // sparse: the flagged probes only
        sray = probe * A.W + k;
        const int px = (int)(probe % A.Px), pz = (int)(probe / A.Px);
        const float2 d = A.dirs[k];
        const float ox = ((float)px + 0.5f) * A.spacing, oz = ((float)pz + 0.5f) * A.spacing;
        const float2* F = A.field + (size_t)lb * A.ncell * LB;

        if constexpr (FIX && HAS_UP) {
            const TS* Rup = reinterpret_cast<const TS*>(A.R_up) + (size_t)lb * A.R_up_lstride;
            fixed_rays<LB, VL, TS>(A, F, Rup, storage_scale<TS>(A, lb), px, pz, ox, oz, d, k,
                                   lane_off, R);
        } else {
            float I[VL], T[VL], I0[VL];
            march_interval<LB, VL>(F, A.nx, A.nz, 0, A.nx, ox, oz, d.x, d.y, A.a, A.b, lane_off,
                                   A.max_steps, I, T, I0);
            if (HAS_UP) {
                const TS* Rup = reinterpret_cast<const TS*>(A.R_up) + (size_t)lb * A.R_up_lstride;
                const Bilinear bl(px, pz, A.Px_up, A.Pz_up);
                const float sc = storage_scale<TS>(A, lb);
                float up[VL];
                upper_radiance<LB, VL, TS>(Rup, bl.b00, bl.b01, bl.b10, bl.b11, bl.fx, bl.fz, A.W,
                                           k, lane_off, up);
#pragma unroll
                for (int j = 0; j < VL; ++j) R[j] = fmaf(T[j], up[j] * sc, I[j]);
            } else {
#pragma unroll
                for (int j = 0; j < VL; ++j) R[j] = I[j];
            }
        }
    }
    store_child_average<LB, VL, TS>(A, lb, valid, sray, lane_off, R);
}

// The group of four sibling rays (consecutive directions of one probe) is summed across
// its lane groups -- LPR lanes apart within a warp, or (more than 8 lanes per ray) spread
// over consecutive warps of the CTA -- and its leader stores the average.  Every thread
// of the CTA calls this.
template <int LB, int VL, typename TS>
__device__ __forceinline__ void store_child_average(const LevelArgs& A, int lb, bool valid,
                                                    long long sray, int lane_off, float (&R)[VL]) {
    constexpr int LPR = LB / VL;
    constexpr int G = 32 / LPR;
    const int g = (threadIdx.x & 31) / LPR;
    bool leader;
    if constexpr (G >= 4) {
#pragma unroll
        for (int j = 0; j < VL; ++j) {
            R[j] += __shfl_xor_sync(0xffffffffu, R[j], LPR);
            R[j] += __shfl_xor_sync(0xffffffffu, R[j], 2 * LPR);
        }
        leader = (g & 3) == 0;
    } else {
        __shared__ float sR[kWarpsPerCta * 32 * VL];
#pragma unroll
        for (int j = 0; j < VL; ++j) sR[threadIdx.x * VL + j] = R[j];
        __syncthreads();
        const int rc = (int)threadIdx.x / LPR;          // ray within the CTA
        leader = (rc & 3) == 0;
        if (leader)
#pragma unroll
            for (int j = 0; j < VL; ++j)
                R[j] = (sR[threadIdx.x * VL + j] + sR[(threadIdx.x + LPR) * VL + j]) +
                       (sR[(threadIdx.x + 2 * LPR) * VL + j] + sR[(threadIdx.x + 3 * LPR) * VL + j]);
    }
    if (valid && leader) {
        TS* out = reinterpret_cast<TS*>(A.R_out) + (size_t)lb * A.R_out_lstride;
        const float inv = __fdividef(0.25f, storage_scale<TS>(A, lb));
#pragma unroll
        for (int j = 0; j < VL; ++j) R[j] *= inv;
        store_vec<TS, VL>(out + (size_t)(sray >> 2) * LB + lane_off, R);
    }
}

template <int LB, int VL, typename TS, bool HAS_UP, bool FIX, bool FAST>
__global__ void __launch_bounds__(kWarpsPerCta * 32, min_ctas<VL>())
level_kernel(const LevelArgs A) {
    level_body<LB, VL, TS, HAS_UP, FIX, FAST>(A, blockIdx.y, blockIdx.x);
}

// The highest launched cascade (no upper) over a list of its CTAs.  A ray that misses the
// box stores 0 there (I = 0 and nothing above it), so the CTAs left out of the list, whose
// rays all miss, are covered by the caller clearing the output first.
template <int LB, int VL, typename TS>
__global__ void __launch_bounds__(kWarpsPerCta * 32, min_ctas<VL>())
level_list_kernel(const LevelArgs A, const int* __restrict__ cta_list) {
    level_body<LB, VL, TS, false, false, true>(A, blockIdx.y, cta_list[blockIdx.x]);
}

// flags[ray / per_cta] = 1 when the ray's interval [a, b] comes within one voxel of the box
// [0, nx] x [0, nz].  FP64 slab test on the march's own probe centre and FP32 direction: the
// FP32 entry test of march_interval errs by far less than the one-voxel margin, so a CTA
// left unflagged has no ray that the march enters the box with.
__global__ void __launch_bounds__(256) top_hits_kernel(const LevelArgs A, int per_cta,
                                                       unsigned char* __restrict__ flags) {
    const long long ray = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= A.rays) return;
    const int k = (int)(ray & (A.W - 1));
    const long long probe = ray >> A.Wshift;
    const int px = (int)(probe % A.Px), pz = (int)(probe / A.Px);
    const float2 d = A.dirs[k];
    const double o[2] = {(double)(((float)px + 0.5f) * A.spacing),
                         (double)(((float)pz + 0.5f) * A.spacing)};
    const double w[2] = {(double)d.x, (double)d.y};
    const double hi[2] = {(double)A.nx + 1.0, (double)A.nz + 1.0};
    double tlo = (double)A.a, thi = (double)A.b;   // b = +inf on the plan's top cascade
    bool miss = false;
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        if (w[ax] == 0.0) {
            miss |= o[ax] < -1.0 || o[ax] > hi[ax];
        } else {
            const double t0 = (-1.0 - o[ax]) / w[ax], t1 = (hi[ax] - o[ax]) / w[ax];
            tlo = fmax(tlo, fmin(t0, t1));
            thi = fmin(thi, fmax(t0, t1));
        }
    }
    if (!miss && tlo <= thi) flags[ray / per_cta] = 1;
}

// ---------------------------------------------------------------------------
// strip-split cascade: when a cascade's rays are long and one lambda block of the field
// does not fit in L2, the domain is cut into n_strips vertical strips and the cascade runs
// as n_strips launches.  Launch p marches, for every ray, only its piece inside strip p, so
// each launch gathers from one strip.  The pieces compose associatively (Eq. 11 applied to
// adjacent pieces): a ray moving to +x meets the strips front to back, I <- I + T I_p,
// T <- T T_p; a ray moving to -x meets them back to front, I <- I_p + T_p I, T <- T_p T.
// The partial (I, T) is kept in it_state between launches; the last launch merges with the
// upper cascade and stores the child averages.
// ---------------------------------------------------------------------------
// FIRST / LAST: this launch is the first / last strip (never both: at least 2 strips).
// FAST as for level_body.
template <int LB, int VL, typename TS, bool HAS_UP, bool FIRST, bool LAST, bool FAST, int WPC>
__global__ void __launch_bounds__(WPC * 32, min_ctas_w<VL, WPC>())
level_split_kernel(const LevelArgs A) {
    constexpr int LPR = LB / VL;
    constexpr int G = 32 / LPR;
    // the merge's group-of-four sum stays within a warp (its shared-memory path is sized for
    // kWarpsPerCta)
    static_assert(G >= 4, "whole groups of four sibling rays per warp");
    const int lane = threadIdx.x & 31;
    const int g = lane / LPR, q = lane % LPR;
    const long long ray = ((long long)blockIdx.x * WPC + (threadIdx.x >> 5)) * G + g;
    const int lane_off = q * VL;
    const int lb = A.split_lb + (int)blockIdx.y;
    const bool valid = ray < A.rays;
    constexpr bool first = FIRST, last = LAST;
    float R[VL];
    long long sray = 0;
#pragma unroll
    for (int j = 0; j < VL; ++j) R[j] = 0.0f;
    if (valid) {
        int k;
        long long probe;
        if (FAST || A.Wshift >= 0) {
            k = (int)(ray & (A.W - 1));
            probe = ray >> A.Wshift;
        } else {
            k = (int)(ray % A.W);
            probe = ray / A.W;
        }
        if (!FAST && A.probe_list) probe = A.probe_list[probe];
        sray = probe * A.W + k;
        int px, pz;
        grid_xy(probe, A.Px, px, pz);
        const float2 d = A.dirs[k];
        const float ox = ((float)px + 0.5f) * A.spacing, oz = ((float)pz + 0.5f) * A.spacing;
        const float2* F = A.field + (size_t)lb * A.ncell * LB;
        float I[VL], T[VL], I0[VL];
        const bool hit = march_interval<LB, VL>(F, A.nx, A.nz, A.strip_x0, A.strip_x1, ox, oz,
                                                d.x, d.y, A.a,
                                                A.b, lane_off, A.max_steps, I, T, I0);
        float2* st = A.it_state + ((size_t)blockIdx.y * A.rays + ray) * LB + lane_off;
        // a ray with no piece in a middle strip leaves its partial (I, T) as it is
        if (hit || first || last) {
            if (!first) {
                const bool forward = d.x >= 0.0f;   // strips met front to back
#pragma unroll
                for (int j = 0; j < VL; ++j) {      // the partial (I, T) of the strips before
                    const float2 acc = st[j];
                    I[j] = forward ? fmaf(acc.y, I[j], acc.x) : fmaf(T[j], acc.x, I[j]);
                    T[j] *= acc.y;
                }
            }
            if (!last) {
#pragma unroll
                for (int j = 0; j < VL; ++j) {
                    // two 32-bit stores (measured 0.3 % faster than one paired store)
                    float* sp = reinterpret_cast<float*>(st + j);
                    asm volatile("st.global.f32 [%0], %1;" :: "l"(sp), "f"(I[j]) : "memory");
                    asm volatile("st.global.f32 [%0], %1;" :: "l"(sp + 1), "f"(T[j]) : "memory");
                }
            } else if (HAS_UP) {
                const TS* Rup = reinterpret_cast<const TS*>(A.R_up) + (size_t)lb * A.R_up_lstride;
                const Bilinear bl(px, pz, A.Px_up, A.Pz_up);
                const float sc = storage_scale<TS>(A, lb);
                float up[VL];
                upper_radiance<LB, VL, TS>(Rup, bl.b00, bl.b01, bl.b10, bl.b11, bl.fx, bl.fz,
                                           A.W, k, lane_off, up);
#pragma unroll
                for (int j = 0; j < VL; ++j) R[j] = fmaf(T[j], up[j] * sc, I[j]);
            } else {
#pragma unroll
                for (int j = 0; j < VL; ++j) R[j] = I[j];
            }
        }
    }
    if (last) store_child_average<LB, VL, TS>(A, lb, valid, sray, lane_off, R);
}

// ---------------------------------------------------------------------------
// shared-DDA march (cascades >= 1, dense plans with a power-of-two direction count).
//
// In the lane-group march above every lane of a ray's group walks the ray's DDA, so a
// warp spends one DDA step's instructions on 32 VL / LB rays.  Here a warp owns 32 rays of
// one lambda block and splits the work in two phases per chunk of kSdSteps steps:
//   * produce: lane r walks the DDA of ray r for the chunk and writes each step's voxel
//     offset and path length ds to shared memory (one DDA step per 32 rays);
//   * replay: the warp integrates the chunk for the rays' LB wavelengths in NP passes of
//     RPP rays, LB / VL lanes per ray, VL wavelengths per lane: per crossing a lane reads
//     the step (a shared load broadcast to the ray's lanes), gathers its wavelengths and
//     applies Eq. 16 -- the same arithmetic as march_interval, so the results are
//     identical to the lane-group march.
// A ray that has left its interval repeats its last voxel with ds = 0 (no contribution)
// until the chunk ends; passes whose rays have all ended are skipped, and the loop ends
// when every ray of the warp has.  The merge with the upper cascade and the child-average
// store follow per pass.  Strip-split cascades (PHASE 1 first, 2 middle, 3 last strip; 0
// unsplit) compose the pieces through it_state as level_split_kernel does.
// ---------------------------------------------------------------------------
// Two warps per CTA at 16 CTAs/SM (64 registers, 12 KB of shared memory per CTA).  Measured at
// 1024^2 x 64 wavelengths: cascades 1 and 2 take 1.33 and 3.05 ms per step with 2-warp CTAs,
// 1.46 and 3.24 with 8-warp CTAs, 1.56 and 3.49 in the lane-group march.
constexpr int kSdWarps = 2;
#ifndef RCX_MIN_CTAS_SD
#define RCX_MIN_CTAS_SD 16
#endif
constexpr int kSdSteps = 8;

// The DDA of one ray over [a, b] clipped to the box [x0, x1] x [0, nz], one step per call
// (the walk of march_interval: same face parameters, exit and step bound).
struct DdaWalk {
    float t, thi, tnx, tnz, kx, kz, tfx, tfz, dtx, dtz;
    int off, dox, doz, left;
    bool alive;

    // Returns false when the interval misses the box (then alive is false and off is 0).
    __device__ __forceinline__ bool init(int LB, int nx, int nz, int x0, int x1, float ox,
                                         float oz, float wx, float wz, float a, float b,
                                         int max_steps) {
        alive = false;
        off = 0;
        const float invx = wx != 0.0f ? 1.0f / wx : 1e30f;
        const float invz = wz != 0.0f ? 1.0f / wz : 1e30f;
        const float tx0 = ((float)x0 - ox) * invx, tx1 = ((float)x1 - ox) * invx;
        const float tz0 = (0.0f - oz) * invz, tz1 = ((float)nz - oz) * invz;
        const float tlo = fmaxf(a, fmaxf(fminf(tx0, tx1), fminf(tz0, tz1)));
        if (!(tlo < fminf(b, fminf(fmaxf(tx0, tx1), fmaxf(tz0, tz1))))) return false;
        const bool upx = wx > 0.0f, upz = wz > 0.0f;
        const float ex = ox + tlo * wx, ez = oz + tlo * wz;
        int ix = (int)floorf(ex), iz = (int)floorf(ez);
        if (!upx && (float)ix == ex) --ix;
        if (!upz && (float)iz == ez) --iz;
        ix = min(max(ix, x0), x1 - 1);
        iz = min(max(iz, 0), nz - 1);
        const float fx0 = (float)(upx ? ix + 1 : ix), fz0 = (float)(upz ? iz + 1 : iz);
        tfx = wx != 0.0f ? (fx0 - ox) * invx : INFINITY;   // as in march_interval
        tfz = wz != 0.0f ? (fz0 - oz) * invz : INFINITY;
        dtx = fabsf(invx);
        dtz = fabsf(invz);
        const float kx_end = (float)(upx ? x1 - 1 - ix : ix - x0);
        const float kz_end = (float)(upz ? nz - 1 - iz : iz);
        thi = fminf(b, fminf(fmaf(kx_end, dtx, tfx), fmaf(kz_end, dtz, tfz)));
        kx = kz = 0.0f;
        tnx = tfx;
        tnz = tfz;
        off = (iz * nx + ix) * LB;
        dox = upx ? LB : -LB;
        doz = upz ? nx * LB : -nx * LB;
        t = tlo;
        left = max_steps;
        alive = max_steps > 0;
        return true;
    }

    // The current step as (voxel offset, ds bits), then the advance; ds = 0 once ended.
    __device__ __forceinline__ int2 next() {
        const bool stepx = tnx <= tnz;
        const float tn = fminf(fminf(tnx, tnz), thi);
        const int2 r = make_int2(off, __float_as_int(alive ? tn - t : 0.0f));
        const bool go = alive && tn < thi && --left > 0;
        if (go) {
            if (stepx) {
                kx += 1.0f;
                tnx = fmaf(kx, dtx, tfx);
                off += dox;
            } else {
                kz += 1.0f;
                tnz = fmaf(kz, dtz, tfz);
                off += doz;
            }
            t = tn;
        }
        alive = go;
        return r;
    }
};

// Eq. 16 for one crossing of VL wavelengths (the update of march_interval).
template <int VL>
__device__ __forceinline__ void cross_voxel(const Voxel<VL>& v, float ds, float (&I)[VL],
                                            float (&T)[VL]) {
#pragma unroll
    for (int j = 0; j < VL; ++j) {
        const float y = v.v[j].x * ds;
        const float e = exp2_neg(y);
        const float om = one_minus_exp2_neg(y, e);
        I[j] = fmaf(T[j] * v.v[j].y, om, I[j]);
        T[j] *= e;
    }
}

template <int LB, int VL, typename TS, bool HAS_UP, int PHASE, int WPC>
__global__ void __launch_bounds__(WPC * 32, RCX_MIN_CTAS_SD)
level_sdda_kernel(const LevelArgs A) {
    static_assert(VL == 4, "the replay keeps a lane's (I, T) as one float4 pair");
    constexpr int LPR = LB / VL;          // lanes per ray in the replay
    constexpr int RPP = 32 / LPR;         // rays per pass
    constexpr int NP = 32 / RPP;          // passes
    constexpr unsigned PASS_MASK = RPP >= 32 ? 0xffffffffu : ((1u << RPP) - 1u);
    constexpr bool SPLIT = PHASE != 0, FIRST = PHASE == 1, LAST = PHASE == 3;
    // per warp: the chunk's steps [step][ray] and the lanes' (I, T) of every pass, kept in
    // shared memory between passes so that a lane holds one pass's state at a time
    __shared__ int2 sbuf[WPC][kSdSteps][32];
    __shared__ float4 sI[WPC][NP][32], sT[WPC][NP][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = lane / LPR, q = lane % LPR, lane_off = q * VL;
    const int lb = SPLIT ? A.split_lb + (int)blockIdx.y : (int)blockIdx.y;
    const long long ray0 = ((long long)blockIdx.x * WPC + w) * 32;
    const float2* F = A.field + (size_t)lb * A.ncell * LB;

    // producer: the DDA of ray ray0 + lane
    DdaWalk walk;
    walk.alive = false;
    walk.off = 0;
    bool hit = false;
    {
        const long long ray = ray0 + lane;
        if (ray < A.rays) {
            const int k = (int)(ray & (A.W - 1));
            int px, pz;
            grid_xy(ray >> A.Wshift, A.Px, px, pz);
            const float2 d = A.dirs[k];
            hit = walk.init(LB, A.nx, A.nz, SPLIT ? A.strip_x0 : 0, SPLIT ? A.strip_x1 : A.nx,
                            ((float)px + 0.5f) * A.spacing, ((float)pz + 0.5f) * A.spacing,
                            d.x, d.y, A.a, A.b, A.max_steps);
        }
    }
    const unsigned hitmask = __ballot_sync(0xffffffffu, hit);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        sI[w][p][lane] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        sT[w][p][lane] = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
    }
    const float2* Fl = F + lane_off;
    int2 (*buf)[32] = sbuf[w];
    unsigned live = __ballot_sync(0xffffffffu, walk.alive);
    while (live) {
#pragma unroll
        for (int s = 0; s < kSdSteps; ++s) buf[s][lane] = walk.next();
        __syncwarp();
#pragma unroll 1
        for (int p = 0; p < NP; ++p) {
            if (!((live >> (p * RPP)) & PASS_MASK)) continue;   // warp-uniform
            const int rp = p * RPP + g;
            float4 i4 = sI[w][p][lane], t4 = sT[w][p][lane];
            float I[VL] = {i4.x, i4.y, i4.z, i4.w}, T[VL] = {t4.x, t4.y, t4.z, t4.w};
            // two gathers ahead: steps s + 1 and s + 2 are in flight while s is integrated
            int2 st[kSdSteps];
#pragma unroll
            for (int s = 0; s < kSdSteps; ++s) st[s] = buf[s][rp];
            Voxel<VL> v0, v1;
            v0.load(Fl + st[0].x);
            v1.load(Fl + st[1].x);
#pragma unroll
            for (int s = 0; s < kSdSteps; ++s) {
                Voxel<VL> v2;
                if (s + 2 < kSdSteps) v2.load(Fl + st[s + 2].x);
                cross_voxel<VL>(v0, __int_as_float(st[s].y), I, T);
                v0 = v1;
                if (s + 2 < kSdSteps) v1 = v2;
            }
            sI[w][p][lane] = make_float4(I[0], I[1], I[2], I[3]);
            sT[w][p][lane] = make_float4(T[0], T[1], T[2], T[3]);
        }
        __syncwarp();
        live = __ballot_sync(0xffffffffu, walk.alive);
    }

    // merge and store, pass by pass (all lanes take part in the sibling sums)
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int rp = p * RPP + g;
        const long long ray = ray0 + rp;
        const bool valid = ray < A.rays;
        float R[VL];
#pragma unroll
        for (int j = 0; j < VL; ++j) R[j] = 0.0f;
        if (valid) {
            const int k = (int)(ray & (A.W - 1));
            int px, pz;
            grid_xy(ray >> A.Wshift, A.Px, px, pz);
            const float4 i4 = sI[w][p][lane], t4 = sT[w][p][lane];
            float Ip[VL] = {i4.x, i4.y, i4.z, i4.w}, Tp[VL] = {t4.x, t4.y, t4.z, t4.w};
            bool merge = !SPLIT;
            if constexpr (SPLIT) {
                float2* st = A.it_state + ((size_t)blockIdx.y * A.rays + ray) * LB + lane_off;
                const bool h = (hitmask >> rp) & 1u;
                if (h || FIRST || LAST) {
                    if constexpr (!FIRST) {
                        const bool forward = A.dirs[k].x >= 0.0f;   // strips met front to back
#pragma unroll
                        for (int j = 0; j < VL; ++j) {
                            const float2 acc = st[j];
                            Ip[j] = forward ? fmaf(acc.y, Ip[j], acc.x) : fmaf(Tp[j], acc.x, Ip[j]);
                            Tp[j] *= acc.y;
                        }
                    }
                    if constexpr (!LAST) {
#pragma unroll
                        for (int j = 0; j < VL; ++j) {
                            float* sp = reinterpret_cast<float*>(st + j);
                            asm volatile("st.global.f32 [%0], %1;" :: "l"(sp), "f"(Ip[j]) : "memory");
                            asm volatile("st.global.f32 [%0], %1;" :: "l"(sp + 1), "f"(Tp[j]) : "memory");
                        }
                    } else {
                        merge = true;
                    }
                }
            }
            if (merge) {
                if constexpr (HAS_UP) {
                    const TS* Rup = reinterpret_cast<const TS*>(A.R_up) + (size_t)lb * A.R_up_lstride;
                    const Bilinear bl(px, pz, A.Px_up, A.Pz_up);
                    const float sc = storage_scale<TS>(A, lb);
                    float up[VL];
                    upper_radiance<LB, VL, TS>(Rup, bl.b00, bl.b01, bl.b10, bl.b11, bl.fx, bl.fz,
                                               A.W, k, lane_off, up);
#pragma unroll
                    for (int j = 0; j < VL; ++j) R[j] = fmaf(Tp[j], up[j] * sc, Ip[j]);
                } else {
#pragma unroll
                    for (int j = 0; j < VL; ++j) R[j] = Ip[j];
                }
            }
        }
        if (!SPLIT || LAST) store_child_average<LB, VL, TS>(A, lb, valid, ray, lane_off, R);
    }
}

// ---------------------------------------------------------------------------
// cascade 0: one lane group per cell centre, loop over the W_0 directions,
// accumulate J (Eq. 1) and the diagonal operator (Eq. 17)
// ---------------------------------------------------------------------------
// OPS: the operator outputs (alo, J_eff, alo_c) may be requested (else J alone); FAST: no
// sparse cell list.  Both known at compile time.
template <int LB, int VL, typename TS, bool HAS_UP, bool FIX = false, bool OPS = true,
          bool FAST = false>
__device__ __forceinline__ void level0_body(const LevelArgs& A, int lb, long long cta) {
    constexpr bool ops = OPS && !FIX;
    constexpr int LPR = LB / VL;
    constexpr int G = 32 / LPR;
    const int lane = threadIdx.x & 31;
    const int g = lane / LPR, q = lane % LPR;
    const long long wid = cta * kWarpsPerCta + (threadIdx.x >> 5);
    long long cell = wid * G + g;
    if (cell >= A.rays) return;                       // rays = cells (or flagged cells) here
    if (!FAST && A.probe_list) cell = A.probe_list[cell];
    int px, pz;
    grid_xy(cell, A.nx, px, pz);
    const float ox = (float)px + 0.5f, oz = (float)pz + 0.5f;
    const float2* F = A.field + (size_t)lb * A.ncell * LB;
    const int lane_off = q * VL;
    const TS* Rup = nullptr;
    float sc = 1.0f;
    if (HAS_UP) {
        Rup = reinterpret_cast<const TS*>(A.R_up) + (size_t)lb * A.R_up_lstride;
        sc = storage_scale<TS>(A, lb);
    }
    Voxel<VL> own;
    if (ops) own.load(F + (size_t)cell * LB + lane_off);
    const Bilinear bl(px, pz, HAS_UP ? A.Px_up : 1, HAS_UP ? A.Pz_up : 1);

    // J = mean of the merged rays; J_eff leaves out the emission of the cell's own
    // centre-to-edge piece (Eq. 19 with a diagonal operator) and is summed without it, so
    // no cancellation; alo = mean(1 - e^{-chi d_k}) (Eq. 17), alo_c = mean(e^{-chi d_k}).
    float Jsum[VL], Jeff[VL], alo_sum[VL], aloc_sum[VL];
#pragma unroll
    for (int j = 0; j < VL; ++j) Jsum[j] = Jeff[j] = alo_sum[j] = aloc_sum[j] = 0.0f;
    for (int k = 0; k < A.W; ++k) {
        const float2 d = A.dirs[k];
        if constexpr (FIX && HAS_UP) {
            // the bilinear fix serves J only (no diagonal operator, no J_eff)
            float R[VL];
            fixed_rays<LB, VL, TS>(A, F, Rup, sc, px, pz, ox, oz, d, k, lane_off, R);
#pragma unroll
            for (int j = 0; j < VL; ++j) Jsum[j] += R[j];
            continue;
        }
        float I[VL], T[VL], I0[VL];
        march_interval<LB, VL, true>(F, A.nx, A.nz, 0, A.nx, ox, oz, d.x, d.y, A.a, A.b, lane_off,
                                     A.max_steps, I, T, I0);
        float up[VL];
        if (HAS_UP)
            upper_radiance<LB, VL, TS>(Rup, bl.b00, bl.b01, bl.b10, bl.b11, bl.fx, bl.fz, A.W, k,
                                       lane_off, up);
#pragma unroll
        for (int j = 0; j < VL; ++j) {
            float Rnl = I[j];
            if (HAS_UP) Rnl = fmaf(T[j], up[j] * sc, I[j]);
            Jsum[j] += Rnl + I0[j];
            if constexpr (ops) {
                Jeff[j] += Rnl;
                const float y = own.v[j].x * (0.5f / fmaxf(fabsf(d.x), fabsf(d.y)));
                const float e = exp2_neg(y);
                alo_sum[j] += one_minus_exp2_neg(y, e);
                aloc_sum[j] += e;
            }
        }
    }
    const float invW = 1.0f / (float)A.W;
#pragma unroll
    for (int j = 0; j < VL; ++j) {
        const int lam = lb * LB + lane_off + j;
        if (lam < A.n_lambda) {
            const size_t o = (size_t)lam * A.ncell + cell;
            A.J[o] = Jsum[j] * invW;
            if constexpr (ops) {
                if (A.alo) A.alo[o] = alo_sum[j] * invW;
                if (A.J_eff) A.J_eff[o] = Jeff[j] * invW;
                if (A.alo_c) A.alo_c[o] = aloc_sum[j] * invW;
            }
        }
    }
}

template <int LB, int VL, typename TS, bool HAS_UP, bool FIX, bool OPS, bool FAST>
__global__ void __launch_bounds__(kWarpsPerCta * 32, OPS ? RCX_MIN_CTAS_L0 : RCX_MIN_CTAS_L0J)
level0_kernel(const LevelArgs A) {
    level0_body<LB, VL, TS, HAS_UP, FIX, OPS, FAST>(A, blockIdx.y, blockIdx.x);
}

// ---------------------------------------------------------------------------
// batched: one launch per cascade over the CTA-sized chunks of every (domain, lambda
// block) segment of a batch, one chunk per CTA, segments sorted by estimated cost (most
// expensive first) so the tail of the launch is made of cheap chunks.  The hardware hands
// out CTAs in index order, which keeps the chunks in flight within a few segments (the
// same L2 footprint as a single-domain launch) and balances uneven chunk costs.
// Chunk t belongs to the last segment whose prefix is <= t; that domain's arguments are
// staged in shared memory.
// ---------------------------------------------------------------------------
template <bool LEVEL0, int LB, int VL, typename TS, bool HAS_UP>
__global__ void __launch_bounds__(kWarpsPerCta * 32, min_ctas<VL>())
batched_level_kernel(const BatchLevelArgs B) {
    static_assert(sizeof(LevelArgs) % sizeof(int) == 0, "LevelArgs is copied word by word");
    __shared__ __align__(16) int sargs[sizeof(LevelArgs) / sizeof(int)];
    __shared__ int s_dom, s_lblk;
    __shared__ long long s_first;
    const long long t = blockIdx.x;
    // The segment holding chunk t is the one non-empty j with prefix[j] <= t < prefix[j+1]:
    // the threads test one segment each, all loads in flight at once (one memory round trip
    // instead of a serial binary search), and the match publishes its segment.
    for (int j = threadIdx.x; j < B.n_seg; j += blockDim.x) {
        const long long lo = B.prefix[j];
        const long long hi = j + 1 < B.n_seg ? B.prefix[j + 1] : B.total;
        const int dom = B.seg_domain[j], lblk = B.seg_lblk[j];
        if (lo <= t && t < hi) {
            s_dom = dom;
            s_lblk = lblk;
            s_first = lo;
        }
    }
    __syncthreads();
    const int* src = reinterpret_cast<const int*>(B.args + s_dom);
    for (int w = threadIdx.x; w < (int)(sizeof(LevelArgs) / sizeof(int)); w += blockDim.x)
        sargs[w] = src[w];
    __syncthreads();
    const LevelArgs& A = *reinterpret_cast<const LevelArgs*>(sargs);
    if (LEVEL0) level0_body<LB, VL, TS, HAS_UP>(A, s_lblk, t - s_first);
    else level_body<LB, VL, TS, HAS_UP>(A, s_lblk, t - s_first);
}

// ---------------------------------------------------------------------------
// emergent intensity along given rays, front to back (Sec. 3.9): a lane group per ray
// ---------------------------------------------------------------------------
template <int LB, bool CONTRIB>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
emergent_kernel(const EmergentArgs A) {
    constexpr int VL = LB < 4 ? LB : 4;
    constexpr int LPR = LB / VL;
    constexpr int G = 32 / LPR;
    const int lane = threadIdx.x & 31;
    const int g = lane / LPR, q = lane % LPR;
    const long long ray = ((long long)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5)) * G + g;
    if (ray >= A.n_rays) return;
    const int lb = blockIdx.y;
    const float4 r = __ldg(reinterpret_cast<const float4*>(A.rays) + ray);
    const float2* F = A.field + (size_t)lb * A.ncell * LB;
    const int lane_off = q * VL;
    const int lam0 = lb * LB + lane_off;
    const int n_valid = max(0, min(VL, A.n_lambda - lam0));
    float I[VL], T[VL], I0[VL];
    march_interval<LB, VL, false, CONTRIB>(F, A.nx, A.nz, 0, A.nx, r.x, r.y, r.z, r.w, 0.0f, INFINITY,
                                           lane_off, A.max_steps, I, T, I0,
                                           CONTRIB ? A.contrib + (size_t)lam0 * A.ncell : nullptr,
                                           n_valid, A.ncell);
#pragma unroll
    for (int j = 0; j < VL; ++j)
        if (j < n_valid) A.I[(size_t)(lam0 + j) * A.n_rays + ray] = I[j];
}

// Emergent intensity without the contribution function, each ray's span inside the box cut
// into K pieces of equal parameter length that neighbouring lane groups march at once (a
// launch of a few ten thousand long rays otherwise holds only a few waves of warps, whose
// tail is the longest rays).  The pieces compose front to back by Eq. 11 applied to
// adjacent pieces, I = I_0 + T_0 (I_1 + T_1 (I_2 + ...)), through shuffles within the warp.
template <int LB, int K>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
emergent_pieces_kernel(const EmergentArgs A) {
    constexpr int VL = 4;
    constexpr int LPR = LB / VL;            // lanes per (ray, piece)
    constexpr int GP = 32 / LPR;            // (ray, piece) groups per warp
    static_assert(LB % VL == 0 && GP % K == 0, "whole rays per warp");
    constexpr int RPW = GP / K;             // rays per warp
    const int lane = threadIdx.x & 31;
    const int grp = lane / LPR, q = lane % LPR;
    const int rw = grp / K, piece = grp % K;
    const long long ray = ((long long)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5)) * RPW + rw;
    const bool valid = ray < A.n_rays;
    const int lb = blockIdx.y;
    const float2* F = A.field + (size_t)lb * A.ncell * LB;
    const int lane_off = q * VL;
    const int lam0 = lb * LB + lane_off;
    float I[VL], T[VL], I0[VL];
#pragma unroll
    for (int j = 0; j < VL; ++j) {
        I[j] = 0.0f;
        T[j] = 1.0f;
    }
    if (valid) {
        const float4 r = __ldg(reinterpret_cast<const float4*>(A.rays) + ray);
        // the ray's span [tlo, thi] inside the box [0, nx] x [0, nz], t >= 0
        const float invx = r.z != 0.0f ? 1.0f / r.z : 1e30f;
        const float invz = r.w != 0.0f ? 1.0f / r.w : 1e30f;
        const float tx0 = (0.0f - r.x) * invx, tx1 = ((float)A.nx - r.x) * invx;
        const float tz0 = (0.0f - r.y) * invz, tz1 = ((float)A.nz - r.y) * invz;
        const float tlo = fmaxf(0.0f, fmaxf(fminf(tx0, tx1), fminf(tz0, tz1)));
        const float thi = fminf(fmaxf(tx0, tx1), fmaxf(tz0, tz1));
        if (tlo < thi) {
            const float len = (thi - tlo) / (float)K;
            const float a = piece == 0 ? 0.0f : fmaf((float)piece, len, tlo);
            const float b = piece == K - 1 ? INFINITY : fmaf((float)(piece + 1), len, tlo);
            march_interval<LB, VL>(F, A.nx, A.nz, 0, A.nx, r.x, r.y, r.z, r.w, a, b, lane_off,
                                   A.max_steps, I, T, I0);
        }
    }
    // compose from the back: R = I_{K-1}; R = I_p + T_p R for p = K-2 .. 0
    const int base = rw * K * LPR + q;
    float R[VL];
#pragma unroll
    for (int j = 0; j < VL; ++j) {
        R[j] = __shfl_sync(0xffffffffu, I[j], base + (K - 1) * LPR);
#pragma unroll
        for (int p = K - 2; p >= 0; --p) {
            const float Ip = __shfl_sync(0xffffffffu, I[j], base + p * LPR);
            const float Tp = __shfl_sync(0xffffffffu, T[j], base + p * LPR);
            R[j] = fmaf(Tp, R[j], Ip);
        }
    }
    if (valid && piece == 0) {
        const int n_valid = max(0, min(VL, A.n_lambda - lam0));
#pragma unroll
        for (int j = 0; j < VL; ++j)
            if (j < n_valid) A.I[(size_t)(lam0 + j) * A.n_rays + ray] = R[j];
    }
}

// ---------------------------------------------------------------------------
// packing [lambda][cell] (chi, eta) -> [lambda block][cell][LB] (chi' = chi voxel log2 e, S)
// ---------------------------------------------------------------------------
// With n_incl > 1 the packed wavelengths are virtual: l' = l n_incl + j carries the
// wavelength l with the opacity scaled by the inclination's 1/sqrt(1 - mu_j^2) (Sec. 3.1:
// same x-z projection, longer path per projected length; S is unchanged).
// A cell's LB wavelengths are split over kPackThreads<LB> neighbouring threads (8 each), so
// a thread holds 8 pairs and more CTAs are resident to keep loads in flight.
template <int LB>
constexpr int kPackThreads = LB >= 8 ? LB / 8 : 1;

template <int LB>
__global__ void __launch_bounds__(256) pack_kernel(const PackArgs P) {
    constexpr int TPC = kPackThreads<LB>, PL = LB / TPC;   // threads per cell, pairs per thread
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long cell = g / TPC;
    const int part = (int)(g % TPC);
    const int lb = blockIdx.y;
    float smax = 0.0f;
    if (cell < P.ncell) {
        // every load of this thread first (2 PL independent requests in flight), then the
        // arithmetic: the divisions' slow-path branches would otherwise hold each
        // wavelength's loads back until the previous one is done
        const bool cell_on = !P.active || P.active[cell];
        const int l0 = lb * LB + part * PL;                 // first (virtual) wavelength
        float chi[PL], eta[PL];
#pragma unroll
        for (int l = 0; l < PL; ++l) {
            const int lam = (l0 + l) / P.n_incl;
            const bool on = cell_on && lam < P.n_lambda;
            chi[l] = on ? __ldg(P.chi + (size_t)lam * P.ncell + cell) : 0.0f;
            eta[l] = on ? __ldg(P.eta + (size_t)lam * P.ncell + cell) : 0.0f;
        }
        float2 v[PL];
#pragma unroll
        for (int l = 0; l < PL; ++l) {
            const int vlam = l0 + l;
            const int lam = vlam / P.n_incl;
            float c = 0.0f, s = 0.0f;
            if (cell_on && lam < P.n_lambda) {
                const float cv = fmaxf(chi[l] * P.voxel, kChiFloor);
                s = (eta[l] * P.voxel) / cv;
                c = cv * kLog2e;
                if (P.incl_r) c *= P.incl_r[vlam - lam * P.n_incl];
                smax = fmaxf(smax, s);
            }
            v[l] = make_float2(c, s);
        }
        float2* o = P.out + ((size_t)lb * P.ncell + cell) * LB + part * PL;
        if constexpr (PL % 4 == 0) {
            // 32-byte stores (the thread's pairs start on a 32-byte boundary): a warp's
            // stores fill whole sectors of consecutive cells
#pragma unroll
            for (int l = 0; l < PL; l += 4)
                asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                             :: "l"(o + l), "f"(v[l].x), "f"(v[l].y), "f"(v[l + 1].x), "f"(v[l + 1].y),
                                "f"(v[l + 2].x), "f"(v[l + 2].y), "f"(v[l + 3].x), "f"(v[l + 3].y)
                             : "memory");
        } else if constexpr (PL % 2 == 0) {
#pragma unroll
            for (int l = 0; l < PL; l += 2)
                reinterpret_cast<float4*>(o)[l / 2] = make_float4(v[l].x, v[l].y, v[l + 1].x, v[l + 1].y);
        } else {
#pragma unroll
            for (int l = 0; l < PL; ++l) o[l] = v[l];
        }
    }
    if (P.smax_bits) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, off));
        if ((threadIdx.x & 31) == 0 && smax > 0.0f)
            atomicMax(P.smax_bits + lb, __float_as_uint(smax));  // S >= 0: bit order = value order
    }
}

// Batched packing: chunk t (256 cells of one (domain, lambda block) segment).
template <int LB>
__global__ void __launch_bounds__(256) batched_pack_kernel(const BatchPackArgs B) {
    for (long long t = blockIdx.x; t < B.total; t += gridDim.x) {
        int lo = 0, hi = B.n_seg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B.prefix[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const PackArgs& P = B.args[B.seg_domain[lo]];
        const int lb = B.seg_lblk[lo];
        const long long cell = (t - B.prefix[lo]) * 256 + threadIdx.x;
        float smax = 0.0f;
        if (cell < P.ncell) {
#pragma unroll
            for (int l = 0; l < LB; l += 2) {
                float4 q;
                float* qq = reinterpret_cast<float*>(&q);
#pragma unroll
                for (int h = 0; h < 2 && l + h < LB; ++h) {
                    const int lam = lb * LB + l + h;
                    float c = 0.0f, sv = 0.0f;
                    if (lam < P.n_lambda) {
                        const float chi = __ldg(P.chi + (size_t)lam * P.ncell + cell);
                        const float eta = __ldg(P.eta + (size_t)lam * P.ncell + cell);
                        const float cv = fmaxf(chi * P.voxel, kChiFloor);
                        sv = (eta * P.voxel) / cv;
                        c = cv * kLog2e;
                        smax = fmaxf(smax, sv);
                    }
                    qq[2 * h] = c;
                    qq[2 * h + 1] = sv;
                }
                float2* o = P.out + ((size_t)lb * P.ncell + cell) * LB;
                if (LB >= 2) reinterpret_cast<float4*>(o)[l / 2] = q;
                else o[0] = make_float2(qq[0], qq[1]);
            }
        }
        if (P.smax_bits) {
            // the 256 cells of a chunk share one segment: warp max, one atomic per warp
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, off));
            if ((threadIdx.x & 31) == 0 && smax > 0.0f)
                atomicMax(P.smax_bits + lb, __float_as_uint(smax));
        }
    }
}

__global__ void flags_seed_kernel(const unsigned char* __restrict__ active,
                                  unsigned char* __restrict__ f0, long long ncell) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) f0[c] = active[c] ? 1 : 0;
}

__global__ void flags_up_kernel(const unsigned char* __restrict__ f, int Px, int Pz,
                                unsigned char* __restrict__ fu, int Pxu, int Pzu) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long long)Px * Pz || !f[p]) return;
    int jx0, jx1, jz0, jz1;
    float fx, fz;
    upper_coord((int)(p % Px), Pxu, jx0, jx1, fx);
    upper_coord((int)(p / Px), Pzu, jz0, jz1, fz);
    fu[(size_t)jz0 * Pxu + jx0] = 1;   // every bracketing parent, zero weights included
    fu[(size_t)jz0 * Pxu + jx1] = 1;
    fu[(size_t)jz1 * Pxu + jx0] = 1;
    fu[(size_t)jz1 * Pxu + jx1] = 1;
}

// One CTA walks the flags in chunks of 1024 and writes the flagged indices in order
// (a block-wide exclusive scan per chunk): deterministic probe order.
__global__ void __launch_bounds__(1024) compact_kernel(const unsigned char* __restrict__ f, long long n,
                                                       int* __restrict__ list, int* __restrict__ n_out) {
    __shared__ int warp_sums[32];
    __shared__ int base;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) base = 0;
    __syncthreads();
    for (long long c0 = 0; c0 < n; c0 += 1024) {
        const long long c = c0 + tid;
        const int flag = (c < n && f[c]) ? 1 : 0;
        const unsigned mask = __ballot_sync(0xffffffffu, flag);
        const int before_in_warp = __popc(mask & ((1u << lane) - 1u));
        if (lane == 0) warp_sums[w] = __popc(mask);
        __syncthreads();
        if (w == 0) {
            const int v = warp_sums[lane];
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            warp_sums[lane] = x - v;                 // exclusive prefix of the warp counts
        }
        __syncthreads();
        if (flag) list[base + warp_sums[w] + before_in_warp] = (int)c;
        __syncthreads();
        if (tid == 1023) base += warp_sums[31] + __popc(mask);   // total of this chunk
        __syncthreads();
    }
    if (tid == 0) *n_out = base;
}

__global__ void incl_reduce_kernel(const float* __restrict__ in, float* __restrict__ out,
                                   int n_lambda, int n_incl, const float* __restrict__ w,
                                   long long ncell) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y;
    if (c >= ncell || l >= n_lambda) return;
    float s = 0.0f;
    for (int j = 0; j < n_incl; ++j) s = fmaf(w[j], in[((size_t)l * n_incl + j) * ncell + c], s);
    out[(size_t)l * ncell + c] = s;
}

__global__ void scales_kernel(int n, const unsigned int* smax_bits, float* scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const float smax = __uint_as_float(smax_bits[i]);
        scale[i] = smax > 0.0f ? smax / kF16Headroom : 1.0f;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int LB>
static cudaError_t pack_t(int n_lblk, const PackArgs& a, cudaStream_t s) {
    dim3 grid((unsigned)((a.ncell * kPackThreads<LB> + 255) / 256), (unsigned)n_lblk);
    pack_kernel<LB><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pack(int LB, int n_lblk, const PackArgs& a, cudaStream_t s) {
    switch (LB) {
        case 1: return pack_t<1>(n_lblk, a, s);
        case 2: return pack_t<2>(n_lblk, a, s);
        case 4: return pack_t<4>(n_lblk, a, s);
        case 8: return pack_t<8>(n_lblk, a, s);
        case 16: return pack_t<16>(n_lblk, a, s);
        case 32: return pack_t<32>(n_lblk, a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_flags_seed(const unsigned char* active, unsigned char* f0, long long ncell,
                              cudaStream_t s) {
    flags_seed_kernel<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(active, f0, ncell);
    return cudaGetLastError();
}

cudaError_t launch_flags_up(const unsigned char* f, int Px, int Pz, unsigned char* fu, int Pxu,
                            int Pzu, cudaStream_t s) {
    const long long n = (long long)Px * Pz;
    flags_up_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, Px, Pz, fu, Pxu, Pzu);
    return cudaGetLastError();
}

cudaError_t launch_compact(const unsigned char* f, long long n, int* list, int* n_out,
                           cudaStream_t s) {
    compact_kernel<<<1, 1024, 0, s>>>(f, n, list, n_out);
    return cudaGetLastError();
}

template <int LB>
static cudaError_t emergent_t(int n_lblk, const EmergentArgs& a, cudaStream_t s) {
    constexpr int VL = LB < 4 ? LB : 4;
    const long long per_cta = (long long)(32 / (LB / VL)) * kWarpsPerCta;
    if constexpr (LB == 16) {
        if (!a.contrib) {
            // 4 pieces per ray: 2 rays per warp
            constexpr int K = 4;
            const long long rays_per_cta = (long long)(32 / (LB / 4) / K) * kWarpsPerCta;
            const dim3 g2((unsigned)((a.n_rays + rays_per_cta - 1) / rays_per_cta), (unsigned)n_lblk);
            emergent_pieces_kernel<LB, K><<<g2, kWarpsPerCta * 32, 0, s>>>(a);
            return cudaGetLastError();
        }
    }
    dim3 grid((unsigned)((a.n_rays + per_cta - 1) / per_cta), (unsigned)n_lblk);
    if (a.contrib) emergent_kernel<LB, true><<<grid, kWarpsPerCta * 32, 0, s>>>(a);
    else emergent_kernel<LB, false><<<grid, kWarpsPerCta * 32, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_emergent(int LB, int n_lblk, const EmergentArgs& a, cudaStream_t s) {
    if (a.n_rays == 0) return cudaSuccess;
    switch (LB) {
        case 1: return emergent_t<1>(n_lblk, a, s);
        case 2: return emergent_t<2>(n_lblk, a, s);
        case 4: return emergent_t<4>(n_lblk, a, s);
        case 8: return emergent_t<8>(n_lblk, a, s);
        case 16: return emergent_t<16>(n_lblk, a, s);
        case 32: return emergent_t<32>(n_lblk, a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_incl_reduce(const float* in, float* out, int n_lambda, int n_incl,
                               const float* w, long long ncell, cudaStream_t s) {
    dim3 grid((unsigned)((ncell + 255) / 256), (unsigned)n_lambda);
    incl_reduce_kernel<<<grid, 256, 0, s>>>(in, out, n_lambda, n_incl, w, ncell);
    return cudaGetLastError();
}

cudaError_t launch_scales(int n_lblk, const unsigned int* smax_bits, float* scale, cudaStream_t s) {
    scales_kernel<<<(n_lblk + 127) / 128, 128, 0, s>>>(n_lblk, smax_bits, scale);
    return cudaGetLastError();
}

template <int LB, int VL, typename TS>
static cudaError_t level_t(bool level0, bool has_up, int n_lblk, const LevelArgs& a,
                           cudaStream_t s) {
    constexpr int G = 32 / (LB / VL);
    const long long items = a.rays;                   // rays, or cascade-0 cells
    if (items == 0) return cudaSuccess;
    const long long per_cta = (long long)G * kWarpsPerCta;
    dim3 grid((unsigned)((items + per_cta - 1) / per_cta), (unsigned)n_lblk);
    dim3 block(kWarpsPerCta * 32);
    const bool fix = a.bilinear_fix != 0;
    if (level0) {
        const bool ops = a.alo || a.J_eff || a.alo_c, dense = !a.probe_list;
        if (has_up && fix) level0_kernel<LB, VL, TS, true, true, false, false><<<grid, block, 0, s>>>(a);
        else if (has_up && !ops && dense)
            level0_kernel<LB, VL, TS, true, false, false, true><<<grid, block, 0, s>>>(a);
        else if (has_up && dense)
            level0_kernel<LB, VL, TS, true, false, true, true><<<grid, block, 0, s>>>(a);
        else if (has_up) level0_kernel<LB, VL, TS, true, false, true, false><<<grid, block, 0, s>>>(a);
        else if (!ops && dense)
            level0_kernel<LB, VL, TS, false, false, false, true><<<grid, block, 0, s>>>(a);
        else level0_kernel<LB, VL, TS, false, false, true, false><<<grid, block, 0, s>>>(a);
    } else {
        const bool fast = a.Wshift >= 0 && !a.probe_list;
        if (has_up && fix) level_kernel<LB, VL, TS, true, true, false><<<grid, block, 0, s>>>(a);
        else if (has_up && fast) level_kernel<LB, VL, TS, true, false, true><<<grid, block, 0, s>>>(a);
        else if (has_up) level_kernel<LB, VL, TS, true, false, false><<<grid, block, 0, s>>>(a);
        else if (fast) level_kernel<LB, VL, TS, false, false, true><<<grid, block, 0, s>>>(a);
        else level_kernel<LB, VL, TS, false, false, false><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int LB, int VL>
static cudaError_t level_p(int precision, bool level0, bool has_up, int n_lblk,
                           const LevelArgs& a, cudaStream_t s) {
    switch (precision) {
        case RC_STORE_F32: return level_t<LB, VL, float>(level0, has_up, n_lblk, a, s);
        case RC_STORE_F16: return level_t<LB, VL, __half>(level0, has_up, n_lblk, a, s);
        case RC_STORE_BF16: return level_t<LB, VL, __nv_bfloat16>(level0, has_up, n_lblk, a, s);
    }
    return cudaErrorInvalidValue;
}

template <int LB>
static cudaError_t level_v(int VL, int precision, bool level0, bool has_up, int n_lblk,
                           const LevelArgs& a, cudaStream_t s) {
    if constexpr (LB >= 8) {
        if (VL == 8) return level_p<LB, 8>(precision, level0, has_up, n_lblk, a, s);
    }
    if constexpr (LB >= 4) {
        if (VL == 4) return level_p<LB, 4>(precision, level0, has_up, n_lblk, a, s);
    }
    if constexpr (LB >= 2) {
        if (VL == 2) return level_p<LB, 2>(precision, level0, has_up, n_lblk, a, s);
    }
    if (VL == 1) return level_p<LB, 1>(precision, level0, has_up, n_lblk, a, s);
    return cudaErrorInvalidValue;
}

template <bool L0, int LB, int VL, typename TS>
static cudaError_t batched_t(bool has_up, const BatchLevelArgs& b, int grid, cudaStream_t s) {
    if (has_up) batched_level_kernel<L0, LB, VL, TS, true><<<grid, kWarpsPerCta * 32, 0, s>>>(b);
    else batched_level_kernel<L0, LB, VL, TS, false><<<grid, kWarpsPerCta * 32, 0, s>>>(b);
    return cudaGetLastError();
}

template <int LB, int VL, typename TS>
static int batched_occ(bool level0, bool has_up) {
    int n = 0;
    const void* f = level0 ? (has_up ? (const void*)batched_level_kernel<true, LB, VL, TS, true>
                                     : (const void*)batched_level_kernel<true, LB, VL, TS, false>)
                           : (has_up ? (const void*)batched_level_kernel<false, LB, VL, TS, true>
                                     : (const void*)batched_level_kernel<false, LB, VL, TS, false>);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kWarpsPerCta * 32, 0);
    return n;
}

template <int LB, int VL>
static cudaError_t batched_p(int precision, bool level0, bool has_up, const BatchLevelArgs& b,
                             int grid, cudaStream_t s, int* occ) {
    switch (precision) {
        case RC_STORE_F32:
            if (occ) { *occ = batched_occ<LB, VL, float>(level0, has_up); return cudaSuccess; }
            return level0 ? batched_t<true, LB, VL, float>(has_up, b, grid, s)
                          : batched_t<false, LB, VL, float>(has_up, b, grid, s);
        case RC_STORE_F16:
            if (occ) { *occ = batched_occ<LB, VL, __half>(level0, has_up); return cudaSuccess; }
            return level0 ? batched_t<true, LB, VL, __half>(has_up, b, grid, s)
                          : batched_t<false, LB, VL, __half>(has_up, b, grid, s);
        case RC_STORE_BF16:
            if (occ) { *occ = batched_occ<LB, VL, __nv_bfloat16>(level0, has_up); return cudaSuccess; }
            return level0 ? batched_t<true, LB, VL, __nv_bfloat16>(has_up, b, grid, s)
                          : batched_t<false, LB, VL, __nv_bfloat16>(has_up, b, grid, s);
    }
    return cudaErrorInvalidValue;
}

// The batched path instantiates the lane layouts the autotuner picks from.
cudaError_t launch_batched_level(int LB, int VL, int precision, bool level0, bool has_up,
                                 const BatchLevelArgs& b, int grid, cudaStream_t s, int* occ) {
    if (LB == 16 && VL == 4) return batched_p<16, 4>(precision, level0, has_up, b, grid, s, occ);
    if (LB == 8 && VL == 4) return batched_p<8, 4>(precision, level0, has_up, b, grid, s, occ);
    if (LB == 8 && VL == 2) return batched_p<8, 2>(precision, level0, has_up, b, grid, s, occ);
    if (LB == 32 && VL == 4) return batched_p<32, 4>(precision, level0, has_up, b, grid, s, occ);
    if (LB == 4 && VL == 4) return batched_p<4, 4>(precision, level0, has_up, b, grid, s, occ);
    if (LB == 4 && VL == 2) return batched_p<4, 2>(precision, level0, has_up, b, grid, s, occ);
    return cudaErrorInvalidValue;
}

cudaError_t launch_batched_pack(int LB, const BatchPackArgs& b, int grid, cudaStream_t s) {
    switch (LB) {
        case 4: batched_pack_kernel<4><<<grid, 256, 0, s>>>(b); break;
        case 8: batched_pack_kernel<8><<<grid, 256, 0, s>>>(b); break;
        case 16: batched_pack_kernel<16><<<grid, 256, 0, s>>>(b); break;
        case 32: batched_pack_kernel<32><<<grid, 256, 0, s>>>(b); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int LB, int VL, typename TS, bool FAST, int WPC>
static cudaError_t split_phase(bool has_up, const LevelArgs& a, cudaStream_t s) {
    constexpr int G = 32 / (LB / VL);
    const long long per_cta = (long long)G * WPC;
    const dim3 grid((unsigned)((a.rays + per_cta - 1) / per_cta), (unsigned)a.split_nblk);
    const dim3 block(WPC * 32);
    const bool first = a.phase == 0, last = a.phase == a.n_strips - 1;
    if (has_up) {
        if (first) level_split_kernel<LB, VL, TS, true, true, false, FAST, WPC><<<grid, block, 0, s>>>(a);
        else if (last) level_split_kernel<LB, VL, TS, true, false, true, FAST, WPC><<<grid, block, 0, s>>>(a);
        else level_split_kernel<LB, VL, TS, true, false, false, FAST, WPC><<<grid, block, 0, s>>>(a);
    } else {
        if (first) level_split_kernel<LB, VL, TS, false, true, false, FAST, WPC><<<grid, block, 0, s>>>(a);
        else if (last) level_split_kernel<LB, VL, TS, false, false, true, FAST, WPC><<<grid, block, 0, s>>>(a);
        else level_split_kernel<LB, VL, TS, false, false, false, FAST, WPC><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int LB, int VL, typename TS>
static cudaError_t level_split_t(bool has_up, const LevelArgs& a, cudaStream_t s) {
    if (a.rays == 0) return cudaSuccess;
    const bool fast = a.Wshift >= 0 && !a.probe_list;
    const bool wide = a.n_strips >= kSplitWideFrom;
    if (fast && wide) return split_phase<LB, VL, TS, true, kSplitWideWarps>(has_up, a, s);
    if (fast) return split_phase<LB, VL, TS, true, kWarpsPerCta>(has_up, a, s);
    if (wide) return split_phase<LB, VL, TS, false, kSplitWideWarps>(has_up, a, s);
    return split_phase<LB, VL, TS, false, kWarpsPerCta>(has_up, a, s);
}

template <int LB, int VL>
static cudaError_t level_split_p(int precision, bool has_up, const LevelArgs& a, cudaStream_t s) {
    switch (precision) {
        case RC_STORE_F32: return level_split_t<LB, VL, float>(has_up, a, s);
        case RC_STORE_F16: return level_split_t<LB, VL, __half>(has_up, a, s);
        case RC_STORE_BF16: return level_split_t<LB, VL, __nv_bfloat16>(has_up, a, s);
    }
    return cudaErrorInvalidValue;
}

// The split march is instantiated for 4 wavelengths per lane and 8-32 per ray, and for 8
// per lane and 16 per ray.
bool level_split_supported(int LB, int VL) {
    return (VL == 4 && (LB == 8 || LB == 16 || LB == 32)) || (VL == 8 && LB == 16);
}

cudaError_t launch_level_split(int LB, int VL, int precision, bool has_up, const LevelArgs& a,
                               cudaStream_t s) {
    if (!level_split_supported(LB, VL) || a.n_strips < 2 || !a.it_state || a.phase < 0 ||
        a.phase >= a.n_strips || a.split_nblk < 0 || a.split_nblk > 65535)
        return cudaErrorInvalidValue;
    LevelArgs b = a;
    b.split_nblk = std::max(1, a.split_nblk);
    b.strip_x0 = (int)((long long)a.phase * a.nx / a.n_strips);
    b.strip_x1 = (int)((long long)(a.phase + 1) * a.nx / a.n_strips);
    if (VL == 8) return level_split_p<16, 8>(precision, has_up, b, s);
    switch (LB) {
        case 8: return level_split_p<8, 4>(precision, has_up, b, s);
        case 16: return level_split_p<16, 4>(precision, has_up, b, s);
        case 32: return level_split_p<32, 4>(precision, has_up, b, s);
    }
    return cudaErrorInvalidValue;
}

template <int LB, int VL, typename TS, int PHASE, int WPC>
static cudaError_t sdda_w(bool has_up, const LevelArgs& a, unsigned nblk, cudaStream_t s) {
    const long long per_cta = 32LL * WPC;
    const dim3 grid((unsigned)((a.rays + per_cta - 1) / per_cta), nblk);
    const dim3 block(WPC * 32);
    if (has_up) level_sdda_kernel<LB, VL, TS, true, PHASE, WPC><<<grid, block, 0, s>>>(a);
    else level_sdda_kernel<LB, VL, TS, false, PHASE, WPC><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <int LB, int VL, typename TS, int PHASE>
static cudaError_t sdda_t(bool has_up, const LevelArgs& a, unsigned nblk, cudaStream_t s) {
    if (a.rays == 0) return cudaSuccess;
    return sdda_w<LB, VL, TS, PHASE, kSdWarps>(has_up, a, nblk, s);
}

template <int LB, int VL, typename TS>
static cudaError_t sdda_phase(bool has_up, int phase, const LevelArgs& a, unsigned nblk,
                              cudaStream_t s) {
    switch (phase) {
        case 0: return sdda_t<LB, VL, TS, 0>(has_up, a, nblk, s);
        case 1: return sdda_t<LB, VL, TS, 1>(has_up, a, nblk, s);
        case 2: return sdda_t<LB, VL, TS, 2>(has_up, a, nblk, s);
        case 3: return sdda_t<LB, VL, TS, 3>(has_up, a, nblk, s);
    }
    return cudaErrorInvalidValue;
}

template <int LB, int VL>
static cudaError_t sdda_p(int precision, bool has_up, int phase, const LevelArgs& a,
                          unsigned nblk, cudaStream_t s) {
    switch (precision) {
        case RC_STORE_F32: return sdda_phase<LB, VL, float>(has_up, phase, a, nblk, s);
        case RC_STORE_F16: return sdda_phase<LB, VL, __half>(has_up, phase, a, nblk, s);
        case RC_STORE_BF16: return sdda_phase<LB, VL, __nv_bfloat16>(has_up, phase, a, nblk, s);
    }
    return cudaErrorInvalidValue;
}

bool level_sdda_supported(int LB, int VL, const LevelArgs& a) {
    return LB == 16 && VL == 4 && a.Wshift >= 0 && !a.probe_list && !a.bilinear_fix;
}

static cudaError_t sdda_dispatch(int LB, int VL, int precision, bool has_up, int phase,
                                 const LevelArgs& a, unsigned nblk, cudaStream_t s) {
    if (!level_sdda_supported(LB, VL, a) || nblk < 1 || nblk > 65535) return cudaErrorInvalidValue;
    return sdda_p<16, 4>(precision, has_up, phase, a, nblk, s);
}

cudaError_t launch_level_sdda(int LB, int VL, int precision, bool has_up, int n_lblk,
                              const LevelArgs& a, cudaStream_t s) {
    return sdda_dispatch(LB, VL, precision, has_up, 0, a, (unsigned)n_lblk, s);
}

cudaError_t launch_level_split_sdda(int LB, int VL, int precision, bool has_up,
                                    const LevelArgs& a, cudaStream_t s) {
    if (a.n_strips < 2 || !a.it_state || a.phase < 0 || a.phase >= a.n_strips ||
        a.split_nblk < 0 || a.split_nblk > 65535)
        return cudaErrorInvalidValue;
    LevelArgs b = a;
    b.split_nblk = std::max(1, a.split_nblk);
    b.strip_x0 = (int)((long long)a.phase * a.nx / a.n_strips);
    b.strip_x1 = (int)((long long)(a.phase + 1) * a.nx / a.n_strips);
    const int phase = a.phase == 0 ? 1 : (a.phase == a.n_strips - 1 ? 3 : 2);
    return sdda_dispatch(LB, VL, precision, has_up, phase, b, (unsigned)b.split_nblk, s);
}

cudaError_t launch_level(int LB, int VL, int precision, bool level0, bool has_up, int n_lblk,
                         const LevelArgs& a, cudaStream_t s) {
    switch (LB) {
        case 1: return level_v<1>(VL, precision, level0, has_up, n_lblk, a, s);
        case 2: return level_v<2>(VL, precision, level0, has_up, n_lblk, a, s);
        case 4: return level_v<4>(VL, precision, level0, has_up, n_lblk, a, s);
        case 8: return level_v<8>(VL, precision, level0, has_up, n_lblk, a, s);
        case 16: return level_v<16>(VL, precision, level0, has_up, n_lblk, a, s);
        case 32: return level_v<32>(VL, precision, level0, has_up, n_lblk, a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_top_hits(const LevelArgs& a, int per_cta, unsigned char* flags,
                            cudaStream_t s) {
    if (a.Wshift < 0 || per_cta < 1) return cudaErrorInvalidValue;
    if (a.rays == 0) return cudaSuccess;
    top_hits_kernel<<<(unsigned)((a.rays + 255) / 256), 256, 0, s>>>(a, per_cta, flags);
    return cudaGetLastError();
}

bool level_list_supported(int LB, int VL, const LevelArgs& a) {
    return LB == 16 && VL == 4 && a.Wshift >= 0 && !a.probe_list && !a.bilinear_fix;
}

cudaError_t launch_level_list(int LB, int VL, int precision, int n_lblk, const LevelArgs& a,
                              const int* cta_list, long long n_cta, cudaStream_t s) {
    if (!level_list_supported(LB, VL, a) || n_cta > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (n_cta == 0) return cudaSuccess;
    const dim3 grid((unsigned)n_cta, (unsigned)n_lblk), block(kWarpsPerCta * 32);
    switch (precision) {
        case RC_STORE_F32: level_list_kernel<16, 4, float><<<grid, block, 0, s>>>(a, cta_list); break;
        case RC_STORE_F16: level_list_kernel<16, 4, __half><<<grid, block, 0, s>>>(a, cta_list); break;
        case RC_STORE_BF16:
            level_list_kernel<16, 4, __nv_bfloat16><<<grid, block, 0, s>>>(a, cta_list);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace rcx
