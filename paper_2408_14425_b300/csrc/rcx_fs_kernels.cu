// rcx_fs_kernels.cu -- sm_103a kernels of the radiance-cascade formal solution.
//
// Work decomposition (one launch per cascade, top cascade first):
//   * The opacity/emissivity slabs are first packed into a wavelength-blocked
//     layout [lambda block][cell][LB] of (chi per voxel, S = eta/chi) pairs, so
//     that the LB lanes of a lane group that march one ray for LB wavelengths
//     read one contiguous 8*LB-byte run per voxel (one 32-byte sector for
//     LB = 4).  A warp holds 32/LB lane groups = 32/LB rays of neighbouring
//     directions of one probe; they walk the grid in near lock-step, so the
//     warp's DDA instructions serve 32 voxel crossings each.
//   * Each lane marches its ray front to back (Sec. 3.2 allows either order)
//     with the piecewise-constant update of Eq. 16 in FP32, keeping the running
//     transmittance T:  I += T S (1 - e^{-dtau}),  T *= e^{-dtau}.
//   * The merge of Sec. 2.3.1 is fused into the same kernel: the lane reads the
//     four child rays of its direction on each of the four bracketing upper
//     probes (one 16-byte vector per probe thanks to the [ray/4][LB][4] layout
//     of the merged intervals), averages them, interpolates bilinearly with the
//     edge clamp of Sec. 2.5 and forms R = I + T * upper (Eq. 11, the nearer
//     interval attenuating the farther one).
//   * Cascade 0 folds the W_0 directions of its probe (a cell centre) into J
//     (Eq. 1) and, optionally, the diagonal operator of Eq. 17.
// No tensor cores: the march is a gather-bound walk, not a contraction.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rcx_internal.h"

namespace rcx {

// ---------------------------------------------------------------------------
// storage of merged intervals
// ---------------------------------------------------------------------------
template <typename TS>
struct Store;

template <>
struct Store<float> {
    static __device__ __forceinline__ float4 load4(const float* p) {
        return __ldg(reinterpret_cast<const float4*>(p));
    }
    static __device__ __forceinline__ void store(float* p, float v) { *p = v; }
};

template <>
struct Store<__half> {
    static __device__ __forceinline__ float4 load4(const __half* p) {
        uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
        __half2 h0 = *reinterpret_cast<__half2*>(&u.x);
        __half2 h1 = *reinterpret_cast<__half2*>(&u.y);
        float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
        return make_float4(f0.x, f0.y, f1.x, f1.y);
    }
    static __device__ __forceinline__ void store(__half* p, float v) { *p = __float2half_rn(v); }
};

template <>
struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float4 load4(const __nv_bfloat16* p) {
        uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
        __nv_bfloat162 h0 = *reinterpret_cast<__nv_bfloat162*>(&u.x);
        __nv_bfloat162 h1 = *reinterpret_cast<__nv_bfloat162*>(&u.y);
        float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
        return make_float4(f0.x, f0.y, f1.x, f1.y);
    }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float v) {
        *p = __float2bfloat16_rn(v);
    }
};

// ---------------------------------------------------------------------------
// one radiance interval
// ---------------------------------------------------------------------------

// 1 - exp(-x) for x >= 0 without cancellation: the Taylor series
// x - x^2/2 + x^3/6 - x^4/24 below x = 1/32 (truncation < x^4/120 relative),
// 1 - e otherwise (e = exp(-x) already computed).
__device__ __forceinline__ float one_minus_exp_neg(float x, float e) {
    float s = x * fmaf(x, fmaf(x, fmaf(x, -1.0f / 24.0f, 1.0f / 6.0f), -0.5f), 1.0f);
    return x < 0.03125f ? s : 1.0f - e;
}

// R_{a,b}(o, w) for wavelength lane `l` of a lambda block.  Front-to-back DDA
// over the uniform grid (Sec. 3.2); face parameters are recomputed from the
// integer cell index each step so no error accumulates along long rays.
template <int LB>
__device__ __forceinline__ void march_interval(const float2* __restrict__ F, int nx, int nz,
                                               float ox, float oz, float wx, float wz,
                                               float a, float b, int l, int max_steps,
                                               float& I, float& T) {
    I = 0.0f;
    T = 1.0f;
    const float invx = wx != 0.0f ? 1.0f / wx : 1e30f;
    const float invz = wz != 0.0f ? 1.0f / wz : 1e30f;
    // clip [a, b] to the domain box (free space outside, Sec. 3.4)
    const float tx0 = (0.0f - ox) * invx, tx1 = ((float)nx - ox) * invx;
    const float tz0 = (0.0f - oz) * invz, tz1 = ((float)nz - oz) * invz;
    const float tlo = fmaxf(a, fmaxf(fminf(tx0, tx1), fminf(tz0, tz1)));
    const float thi = fminf(b, fminf(fmaxf(tx0, tx1), fmaxf(tz0, tz1)));
    if (!(tlo < thi)) return;

    const int px = wx > 0.0f ? 1 : 0, pz = wz > 0.0f ? 1 : 0;
    const int sx = px ? 1 : -1, sz = pz ? 1 : -1;
    const float ex = ox + tlo * wx, ez = oz + tlo * wz;
    int ix = (int)floorf(ex), iz = (int)floorf(ez);
    if (!px && (float)ix == ex) --ix;   // entering through a face while moving down
    if (!pz && (float)iz == ez) --iz;
    ix = min(max(ix, 0), nx - 1);
    iz = min(max(iz, 0), nz - 1);

    float tnx = ((float)(ix + px) - ox) * invx;
    float tnz = ((float)(iz + pz) - oz) * invz;
    float t = tlo;
    for (int step = 0; step < max_steps; ++step) {
        const float tn = fminf(fminf(tnx, tnz), thi);
        const float ds = fmaxf(tn - t, 0.0f);
        const float2 f = __ldg(F + ((size_t)iz * nx + ix) * LB + l);
        const float dtau = f.x * ds;
        const float e = __expf(-dtau);
        const float om = one_minus_exp_neg(dtau, e);
        I = fmaf(T * f.y, om, I);
        T *= e;
        if (tn >= thi) break;
        if (tnx <= tnz) {
            ix += sx;
            tnx = ((float)(ix + px) - ox) * invx;
        } else {
            iz += sz;
            tnz = ((float)(iz + pz) - oz) * invz;
        }
        if ((unsigned)ix >= (unsigned)nx || (unsigned)iz >= (unsigned)nz) break;
        t = tn;
    }
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

// Child-cone average of the four bracketing upper probes, bilinearly weighted.
template <int LB, typename TS>
__device__ __forceinline__ float upper_radiance(const TS* __restrict__ Rup, int Px_up, int Pz_up,
                                                int px, int pz, int W, int k, int l) {
    int jx0, jx1, jz0, jz1;
    float fx, fz;
    upper_coord(px, Px_up, jx0, jx1, fx);
    upper_coord(pz, Pz_up, jz0, jz1, fz);
    const long long b00 = (long long)jz0 * Px_up + jx0, b01 = (long long)jz0 * Px_up + jx1;
    const long long b10 = (long long)jz1 * Px_up + jx0, b11 = (long long)jz1 * Px_up + jx1;
    // children 4k..4k+3 of probe b sit at [(b W + k) LB + l][0..3]
    const float4 c00 = Store<TS>::load4(Rup + ((size_t)(b00 * W + k) * LB + l) * 4);
    const float4 c01 = Store<TS>::load4(Rup + ((size_t)(b01 * W + k) * LB + l) * 4);
    const float4 c10 = Store<TS>::load4(Rup + ((size_t)(b10 * W + k) * LB + l) * 4);
    const float4 c11 = Store<TS>::load4(Rup + ((size_t)(b11 * W + k) * LB + l) * 4);
    const float s00 = (c00.x + c00.y) + (c00.z + c00.w);
    const float s01 = (c01.x + c01.y) + (c01.z + c01.w);
    const float s10 = (c10.x + c10.y) + (c10.z + c10.w);
    const float s11 = (c11.x + c11.y) + (c11.z + c11.w);
    const float r0 = fmaf(fx, s01 - s00, s00);
    const float r1 = fmaf(fx, s11 - s10, s10);
    return 0.25f * fmaf(fz, r1 - r0, r0);
}

// ---------------------------------------------------------------------------
// cascades >= 1: march + merge, store the merged interval
// ---------------------------------------------------------------------------
template <int LB, typename TS, bool HAS_UP>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
level_kernel(const LevelArgs A) {
    constexpr int G = 32 / LB;
    const int lane = threadIdx.x & 31;
    const int g = lane / LB, l = lane % LB;
    const long long wid = (long long)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
    const long long ray = wid * G + g;
    if (ray >= A.rays) return;
    const int lb = blockIdx.y;

    int k;
    long long probe;
    if (A.Wshift >= 0) {
        k = (int)(ray & (A.W - 1));
        probe = ray >> A.Wshift;
    } else {
        k = (int)(ray % A.W);
        probe = ray / A.W;
    }
    const int px = (int)(probe % A.Px), pz = (int)(probe / A.Px);
    const float2 d = A.dirs[k];
    const float ox = ((float)px + 0.5f) * A.spacing, oz = ((float)pz + 0.5f) * A.spacing;
    const float2* F = A.field + (size_t)lb * A.ncell * LB;

    float I, T;
    march_interval<LB>(F, A.nx, A.nz, ox, oz, d.x, d.y, A.a, A.b, l, A.max_steps, I, T);
    float R = I;
    if (HAS_UP) {
        const TS* Rup = reinterpret_cast<const TS*>(A.R_up) + (size_t)lb * A.R_up_lstride;
        float up = upper_radiance<LB, TS>(Rup, A.Px_up, A.Pz_up, px, pz, A.W, k, l);
        if (A.scale) up *= A.scale[lb];
        R = fmaf(T, up, I);
    }
    TS* out = reinterpret_cast<TS*>(A.R_out) + (size_t)lb * A.R_out_lstride;
    const float inv = A.scale ? 1.0f / A.scale[lb] : 1.0f;
    Store<TS>::store(out + ((size_t)(ray >> 2) * LB + l) * 4 + (ray & 3), R * inv);
}

// ---------------------------------------------------------------------------
// cascade 0: one lane group per cell centre, loop over the W_0 directions,
// accumulate J (Eq. 1) and the diagonal operator (Eq. 17)
// ---------------------------------------------------------------------------
template <int LB, typename TS, bool HAS_UP>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
level0_kernel(const LevelArgs A) {
    constexpr int G = 32 / LB;
    const int lane = threadIdx.x & 31;
    const int g = lane / LB, l = lane % LB;
    const long long wid = (long long)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
    const long long cell = wid * G + g;
    if (cell >= A.ncell) return;
    const int lb = blockIdx.y;
    const int px = (int)(cell % A.nx), pz = (int)(cell / A.nx);
    const float ox = (float)px + 0.5f, oz = (float)pz + 0.5f;
    const float2* F = A.field + (size_t)lb * A.ncell * LB;
    const TS* Rup = nullptr;
    float up_scale = 1.0f;
    if (HAS_UP) {
        Rup = reinterpret_cast<const TS*>(A.R_up) + (size_t)lb * A.R_up_lstride;
        if (A.scale) up_scale = A.scale[lb];
    }
    const float chi_c = __ldg(F + (size_t)cell * LB + l).x;

    float Jsum = 0.0f, alo_sum = 0.0f;
    for (int k = 0; k < A.W; ++k) {
        const float2 d = A.dirs[k];
        float I, T;
        march_interval<LB>(F, A.nx, A.nz, ox, oz, d.x, d.y, A.a, A.b, l, A.max_steps, I, T);
        float R = I;
        if (HAS_UP) {
            const float up = upper_radiance<LB, TS>(Rup, A.Px_up, A.Pz_up, px, pz, A.W, k, l);
            R = fmaf(T, up * up_scale, I);
        }
        Jsum += R;
        const float dk = 0.5f / fmaxf(fabsf(d.x), fabsf(d.y));
        const float x = chi_c * dk;
        alo_sum += one_minus_exp_neg(x, __expf(-x));
    }
    const int lam = lb * LB + l;
    if (lam < A.n_lambda) {
        const float invW = 1.0f / (float)A.W;
        A.J[(size_t)lam * A.ncell + cell] = Jsum * invW;
        if (A.alo) A.alo[(size_t)lam * A.ncell + cell] = alo_sum * invW;
    }
}

// ---------------------------------------------------------------------------
// packing [lambda][cell] (chi, eta) -> [lambda block][cell][LB] (chi_vox, S)
// ---------------------------------------------------------------------------
template <int LB>
__global__ void __launch_bounds__(256) pack_kernel(const PackArgs P) {
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lb = blockIdx.y;
    float smax = 0.0f;
    if (cell < P.ncell) {
        float2 v[LB];
#pragma unroll
        for (int l = 0; l < LB; ++l) {
            const int lam = lb * LB + l;
            float c = 0.0f, s = 0.0f;
            if (lam < P.n_lambda) {
                const float chi = __ldg(P.chi + (size_t)lam * P.ncell + cell);
                const float eta = __ldg(P.eta + (size_t)lam * P.ncell + cell);
                c = fmaxf(chi * P.voxel, kChiFloor);
                s = (eta * P.voxel) / c;
                smax = fmaxf(smax, s);
            }
            v[l] = make_float2(c, s);
        }
        float2* o = P.out + ((size_t)lb * P.ncell + cell) * LB;
        if constexpr (LB % 2 == 0) {
#pragma unroll
            for (int l = 0; l < LB; l += 2)
                reinterpret_cast<float4*>(o)[l / 2] = make_float4(v[l].x, v[l].y, v[l + 1].x, v[l + 1].y);
        } else {
#pragma unroll
            for (int l = 0; l < LB; ++l) o[l] = v[l];
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
    dim3 grid((unsigned)((a.ncell + 255) / 256), (unsigned)n_lblk);
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

cudaError_t launch_scales(int n_lblk, const unsigned int* smax_bits, float* scale, cudaStream_t s) {
    scales_kernel<<<(n_lblk + 127) / 128, 128, 0, s>>>(n_lblk, smax_bits, scale);
    return cudaGetLastError();
}

template <int LB, typename TS>
static cudaError_t level_t(bool level0, bool has_up, int n_lblk, const LevelArgs& a,
                           cudaStream_t s) {
    constexpr int G = 32 / LB;
    const long long items = level0 ? a.ncell : a.rays;
    const long long per_cta = (long long)G * kWarpsPerCta;
    dim3 grid((unsigned)((items + per_cta - 1) / per_cta), (unsigned)n_lblk);
    dim3 block(kWarpsPerCta * 32);
    if (level0) {
        if (has_up) level0_kernel<LB, TS, true><<<grid, block, 0, s>>>(a);
        else level0_kernel<LB, TS, false><<<grid, block, 0, s>>>(a);
    } else {
        if (has_up) level_kernel<LB, TS, true><<<grid, block, 0, s>>>(a);
        else level_kernel<LB, TS, false><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int LB>
static cudaError_t level_p(int precision, bool level0, bool has_up, int n_lblk,
                           const LevelArgs& a, cudaStream_t s) {
    switch (precision) {
        case RC_STORE_F32: return level_t<LB, float>(level0, has_up, n_lblk, a, s);
        case RC_STORE_F16: return level_t<LB, __half>(level0, has_up, n_lblk, a, s);
        case RC_STORE_BF16: return level_t<LB, __nv_bfloat16>(level0, has_up, n_lblk, a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_level(int LB, int precision, bool level0, bool has_up, int n_lblk,
                         const LevelArgs& a, cudaStream_t s) {
    switch (LB) {
        case 1: return level_p<1>(precision, level0, has_up, n_lblk, a, s);
        case 2: return level_p<2>(precision, level0, has_up, n_lblk, a, s);
        case 4: return level_p<4>(precision, level0, has_up, n_lblk, a, s);
        case 8: return level_p<8>(precision, level0, has_up, n_lblk, a, s);
        case 16: return level_p<16>(precision, level0, has_up, n_lblk, a, s);
        case 32: return level_p<32>(precision, level0, has_up, n_lblk, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rcx
