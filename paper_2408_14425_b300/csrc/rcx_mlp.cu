// rcx_mlp.cu -- the surrogate network that seeds the non-LTE iteration: a 6-64-64-3
// tanh MLP with input standardisation, trained and run by these kernels.  The paper has
// no learned component; the iteration it seeds is Sec. 3.3's.
//
// Precision: master weights and Adam moments in FP32; the forward and backward passes
// multiply with the bfloat16-rounded weights and accumulate in FP32.
// Work layout: one CTA of 256 threads per tile of 128 samples holds the weights and the
// tile's activations in shared memory (about 150 KB) and runs the forward pass, the loss
// and (for training) the whole backward pass; weight gradients are summed over the tile
// and stored as the tile's partial gradient, which a second kernel sums over the tiles in
// a fixed order, so training is bit-for-bit reproducible.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "rcx_internal.h"

namespace {

constexpr int NI = 6, NH = 64, NO = 3;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NI, OFF_W2 = OFF_B1 + NH;
constexpr int OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH;
constexpr int NPARAM = OFF_B3 + NO;
constexpr int TILE = 128;
constexpr int THREADS = 256;
constexpr int LD = NH + 1;   // padded row of an activation tile

struct Smem {
    float w[NPARAM];          // bf16-rounded weights, [out][in]
    float w2t[NH * NH];       // W2 transposed: [in][out]
    float mean[NI], istd[NI];
    float xn[TILE * NI];
    float h1[TILE * LD];
    float h2[TILE * LD];      // becomes dh1 in the backward pass
    float d[TILE * LD];       // dh2
    float dy[TILE * NO];
    float red[THREADS / 32];
};

rc_status mfail(rc_status s, const std::string& m) {
    rcx::set_last_error(m);
    return s;
}
rc_status mcuda(cudaError_t e, const char* what) {
    cudaGetLastError();
    rcx::set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    return RC_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// fused forward (+ loss, + backward) over one tile of samples
// ---------------------------------------------------------------------------
template <bool TRAIN>
__global__ void __launch_bounds__(THREADS)
mlp_tile_kernel(const float* __restrict__ wbf, const float* __restrict__ norm,
                const float* __restrict__ X, const float* __restrict__ Yt, long long B,
                float* __restrict__ Y, float* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // this tile's partial gradient [NPARAM] and loss (training only)
    float* const grad = TRAIN ? part + (size_t)blockIdx.x * (NPARAM + 1) : nullptr;
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    const int tid = threadIdx.x;
    const long long s0 = (long long)blockIdx.x * TILE;
    const int nvalid = (int)min((long long)TILE, B - s0);

    for (int i = tid; i < NPARAM; i += THREADS) S.w[i] = wbf[i];
    for (int i = tid; i < NH * NH; i += THREADS) {
        const int o = i / NH, k = i % NH;
        S.w2t[k * NH + o] = wbf[OFF_W2 + i];
    }
    if (tid < NI) {
        S.mean[tid] = norm[tid];
        S.istd[tid] = 1.0f / norm[NI + tid];
    }
    __syncthreads();
    for (int i = tid; i < TILE * NI; i += THREADS) {
        const int s = i / NI, f = i % NI;
        S.xn[i] = s < nvalid ? (X[(s0 + s) * NI + f] - S.mean[f]) * S.istd[f] : 0.0f;
    }
    __syncthreads();
    // h1 = tanh(W1 xn + b1)
    for (int i = tid; i < TILE * NH; i += THREADS) {
        const int s = i / NH, o = i % NH;
        float a = S.w[OFF_B1 + o];
#pragma unroll
        for (int f = 0; f < NI; ++f) a = fmaf(S.w[OFF_W1 + o * NI + f], S.xn[s * NI + f], a);
        S.h1[s * LD + o] = tanhf(a);
    }
    __syncthreads();
    // h2 = tanh(W2 h1 + b2): each thread a 4-sample x 8-output block
    {
        const int sg = tid / 8, og = tid % 8;
        const int sb = sg * 4, ob = og * 8;
        float acc[4][8];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] = S.w[OFF_B2 + ob + c];
        for (int k = 0; k < NH; ++k) {
            float a[4], w[8];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = S.h1[(sb + r) * LD + k];
#pragma unroll
            for (int c = 0; c < 8; ++c) w[c] = S.w2t[k * NH + ob + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], w[c], acc[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) S.h2[(sb + r) * LD + ob + c] = tanhf(acc[r][c]);
    }
    __syncthreads();
    // y = W3 h2 + b3, loss, dy
    float lsum = 0.0f;
    for (int i = tid; i < TILE * NO; i += THREADS) {
        const int s = i / NO, o = i % NO;
        float a = S.w[OFF_B3 + o];
        for (int k = 0; k < NH; ++k) a = fmaf(S.w[OFF_W3 + o * NH + k], S.h2[s * LD + k], a);
        if (s < nvalid) {
            if (Y) Y[(s0 + s) * NO + o] = a;
            if (TRAIN) {
                const float r = a - Yt[(s0 + s) * NO + o];
                lsum += r * r;
                S.dy[i] = 2.0f * r / (float)(B * NO);
            }
        } else if (TRAIN) {
            S.dy[i] = 0.0f;
        }
    }
    if constexpr (TRAIN) {
    // loss: block sum
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((tid & 31) == 0) S.red[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
        float t = 0.0f;
        for (int w = 0; w < THREADS / 32; ++w) t += S.red[w];
        grad[NPARAM] = t / (float)(B * NO);
    }
    // dW3, db3
    if (tid < NO * NH) {
        const int o = tid / NH, k = tid % NH;
        float g = 0.0f;
        for (int s = 0; s < TILE; ++s) g = fmaf(S.dy[s * NO + o], S.h2[s * LD + k], g);
        grad[OFF_W3 + tid] = g;
    } else if (tid < NO * NH + NO) {
        const int o = tid - NO * NH;
        float g = 0.0f;
        for (int s = 0; s < TILE; ++s) g += S.dy[s * NO + o];
        grad[OFF_B3 + o] = g;
    }
    // dh2 = (W3^T dy) * (1 - h2^2)
    for (int i = tid; i < TILE * NH; i += THREADS) {
        const int s = i / NH, k = i % NH;
        float a = 0.0f;
#pragma unroll
        for (int o = 0; o < NO; ++o) a = fmaf(S.dy[s * NO + o], S.w[OFF_W3 + o * NH + k], a);
        const float h = S.h2[s * LD + k];
        S.d[s * LD + k] = a * (1.0f - h * h);
    }
    __syncthreads();
    // dW2[o][k] = sum_s dh2[s][o] h1[s][k]: each thread a 4 x 4 block; db2
    {
        const int ob = (tid / 16) * 4, kb = (tid % 16) * 4;
        float g[4][4] = {};
        for (int s = 0; s < TILE; ++s) {
            float dv[4], hv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) dv[r] = S.d[s * LD + ob + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) hv[c] = S.h1[s * LD + kb + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) g[r][c] = fmaf(dv[r], hv[c], g[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) grad[OFF_W2 + (ob + r) * NH + kb + c] = g[r][c];
        if (tid < NH) {
            float gb = 0.0f;
            for (int s = 0; s < TILE; ++s) gb += S.d[s * LD + tid];
            grad[OFF_B2 + tid] = gb;
        }
    }
    __syncthreads();
    // dh1 = (W2^T dh2) * (1 - h1^2), written over h2
    {
        const int sg = tid / 8, ig = tid % 8;
        const int sb = sg * 4, ib = ig * 8;
        float acc[4][8] = {};
        for (int o = 0; o < NH; ++o) {
            float a[4], w[8];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = S.d[(sb + r) * LD + o];
#pragma unroll
            for (int c = 0; c < 8; ++c) w[c] = S.w[OFF_W2 + o * NH + ib + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], w[c], acc[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float h = S.h1[(sb + r) * LD + ib + c];
                S.h2[(sb + r) * LD + ib + c] = acc[r][c] * (1.0f - h * h);
            }
    }
    __syncthreads();
    // dW1[o][f] = sum_s dh1[s][o] xn[s][f]; db1
    for (int i = tid; i < NH * NI + NH; i += THREADS) {
        if (i < NH * NI) {
            const int o = i / NI, f = i % NI;
            float g = 0.0f;
            for (int s = 0; s < TILE; ++s) g = fmaf(S.h2[s * LD + o], S.xn[s * NI + f], g);
            grad[OFF_W1 + i] = g;
        } else {
            const int o = i - NH * NI;
            float g = 0.0f;
            for (int s = 0; s < TILE; ++s) g += S.h2[s * LD + o];
            grad[OFF_B1 + o] = g;
        }
    }
    }  // TRAIN
}

// ---------------------------------------------------------------------------
// inference with the 64 x 64 layer on the tensor cores (tcgen05, sm_100 family)
//
// Per CTA of 128 samples: h1 (128 x 64) and W2 (64 x 64) as bf16 in shared memory in the
// no-swizzle K-major layout of 8-row x 16-byte core matrices (K step between core matrices
// 128 B, row-group step 1024 B); one elected thread issues four tcgen05.mma (M = 128,
// N = 64, K = 16 each, FP32 accumulation in 64 TMEM columns) and commits them to an
// mbarrier; every warp waits (bounded) and reads its quarter of the rows back with
// tcgen05.ld for the bias, tanh and the 64 -> 3 output layer.
// ---------------------------------------------------------------------------
constexpr int TC_SMEM_A = TILE * NH * 2;     // 16 KB bf16
constexpr int TC_SMEM_B = NH * NH * 2;       //  8 KB bf16
constexpr unsigned kTcWaitLimit = 1u << 21;  // mbarrier polls before giving up

struct TcSmem {
    alignas(1024) unsigned char a[TC_SMEM_A];
    alignas(1024) unsigned char b[TC_SMEM_B];
    float w1[NH * NI], b1[NH], b2[NH], w3[NO * NH], b3[NO];
    float mean[NI], istd[NI];
    float part[2][TILE][NO];   // output layer over each half of h2's columns
    alignas(8) unsigned long long mbar;
    unsigned tmem_base;
};

// byte offset of element (row r, k) of a K-major no-swizzle operand with K = 64
__device__ __forceinline__ int core_offset(int r, int k) {
    return (r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// Waits for phase `parity` of the mbarrier at shared address `mbar` with non-blocking polls
// and a short sleep between them, at most `limit` polls (about limit x 64 ns); false if it
// gave up.  Every device-side wait of this library goes through here.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned mbar, unsigned parity, unsigned limit) {
    for (unsigned it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile("{\n\t.reg .pred q;\n\t"
                     "mbarrier.test_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, q;\n\t}"
                     : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
        __nanosleep(64);
    }
    return false;
}

// Self-test of the bounded wait: an mbarrier that expects one arrival nobody makes.  The
// wait must give up after `limit` polls and report it; the context stays usable.
__global__ void wait_timeout_probe_kernel(unsigned limit, int* __restrict__ timed_out) {
    __shared__ __align__(8) unsigned long long bar;
    const unsigned mb = (unsigned)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    __syncthreads();
    const bool ok = mbar_wait_bounded(mb, 0, limit);
    if (threadIdx.x == 0) *timed_out = ok ? 0 : 1;
}

__device__ __forceinline__ unsigned long long smem_desc(const void* p) {
    const unsigned addr = (unsigned)__cvta_generic_to_shared(p);
    unsigned long long d = 0;
    d |= (unsigned long long)((addr >> 4) & 0x3FFF);          // start address
    d |= (unsigned long long)((128 >> 4) & 0x3FFF) << 16;      // leading (K) byte offset
    d |= (unsigned long long)((1024 >> 4) & 0x3FFF) << 32;     // stride (row group) byte offset
    d |= 1ull << 46;                                           // descriptor version (sm_100)
    return d;                                                  // base offset 0, no swizzle
}

// instruction descriptor: FP32 accumulate, bf16 A and B, both K-major, N = 64, M = 128
__device__ __forceinline__ unsigned mma_idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(NH >> 3) << 17) |
           ((unsigned)(TILE >> 4) << 24);
}

__global__ void __launch_bounds__(THREADS)
mlp_forward_tc_kernel(const float* __restrict__ wbf, const float* __restrict__ norm,
                      const float* __restrict__ X, long long B, float* __restrict__ Y,
                      int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    // the launch adds 1024 B of slack so the operand tiles can start on a 1024 B boundary
    const unsigned raw_s = (unsigned)__cvta_generic_to_shared(tc_raw);
    TcSmem& S = *reinterpret_cast<TcSmem*>(tc_raw + (((raw_s + 1023u) & ~1023u) - raw_s));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long s0 = (long long)blockIdx.x * TILE;
    const int nvalid = (int)min((long long)TILE, B - s0);

    if (warp == 0) {   // TMEM: 64 columns for the 128 x 64 FP32 accumulator
        const unsigned dst = (unsigned)__cvta_generic_to_shared(&S.tmem_base);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(dst));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        const unsigned mb = (unsigned)__cvta_generic_to_shared(&S.mbar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    }
    for (int i = tid; i < NH * NI; i += THREADS) S.w1[i] = wbf[OFF_W1 + i];
    for (int i = tid; i < NH; i += THREADS) {
        S.b1[i] = wbf[OFF_B1 + i];
        S.b2[i] = wbf[OFF_B2 + i];
    }
    for (int i = tid; i < NO * NH; i += THREADS) S.w3[i] = wbf[OFF_W3 + i];
    if (tid < NO) S.b3[tid] = wbf[OFF_B3 + tid];
    if (tid < NI) {
        S.mean[tid] = norm[tid];
        S.istd[tid] = 1.0f / norm[NI + tid];
    }
    // W2 [out n][in k] is already K-major for D[m][n] = sum_k A[m][k] B[n][k]; four
    // consecutive k of a row share one 8-byte row of a core matrix
    for (int i = tid; i < NH * NH / 4; i += THREADS) {
        const int n = (4 * i) / NH, k = (4 * i) % NH;
        const float* w = wbf + OFF_W2 + 4 * i;
        const __nv_bfloat162 lo = __floats2bfloat162_rn(w[0], w[1]);
        const __nv_bfloat162 hi = __floats2bfloat162_rn(w[2], w[3]);
        *reinterpret_cast<uint2*>(S.b + core_offset(n, k)) =
            make_uint2(*reinterpret_cast<const unsigned*>(&lo), *reinterpret_cast<const unsigned*>(&hi));
    }
    __syncthreads();
    // h1 = tanh(W1 xn + b1) as bf16 into the A operand: two threads per sample, 32 outputs
    // each, the sample's standardised inputs computed once
    {
        static_assert(THREADS == 2 * TILE, "two threads per sample row");
        const int r = tid >> 1, obase = (tid & 1) * (NH / 2);
        const bool rv = r < nvalid;
        float xn[NI];
#pragma unroll
        for (int f = 0; f < NI; ++f) xn[f] = rv ? (X[(s0 + r) * NI + f] - S.mean[f]) * S.istd[f] : 0.0f;
#pragma unroll 4
        for (int o = obase; o < obase + NH / 2; o += 2) {
            float h[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                float a = 0.0f;
                if (rv) {
                    a = S.b1[o + q];
#pragma unroll
                    for (int f = 0; f < NI; ++f) a = fmaf(S.w1[(o + q) * NI + f], xn[f], a);
                    a = tanhf(a);
                }
                h[q] = a;
            }
            *reinterpret_cast<__nv_bfloat162*>(S.a + core_offset(r, o)) = __floats2bfloat162_rn(h[0], h[1]);
        }
    }
    // generic-proxy stores -> visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = S.tmem_base;
    const unsigned mb = (unsigned)__cvta_generic_to_shared(&S.mbar);
    if (tid == 0) {
        const unsigned idesc = mma_idesc();
#pragma unroll
        for (int kk = 0; kk < NH / 16; ++kk) {
            // K = 16 per instruction: advance both operands by two core matrices (256 B)
            const unsigned long long da = smem_desc(S.a + kk * 256);
            const unsigned long long db = smem_desc(S.b + kk * 256);
            const unsigned acc = kk > 0 ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(mb) : "memory");
    }
    // bounded wait for the MMAs (phase 0); block-uniform outcome: the epilogue's
    // .sync.aligned loads need whole warps
    unsigned done = mbar_wait_bounded(mb, 0, kTcWaitLimit) ? 1u : 0u;
    done = __syncthreads_and(done);
    if (!done && tid == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: warp w reads rows 32 (w % 4) .. +31 and columns 32 (w / 4) .. +31
    if (done) {
        const int rbase = 32 * (warp & 3), cbase = 32 * (warp >> 2);
        unsigned v[32];
        const unsigned taddr = tmem + ((unsigned)rbase << 16) + (unsigned)cbase;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
              "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
              "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
              "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // h2 = tanh(D + b2) stays in registers: this warp's share of the 64 -> 3 layer
        const int r = rbase + lane;
        float p[NO] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const float h = tanhf(__uint_as_float(v[c]) + S.b2[cbase + c]);
#pragma unroll
            for (int o = 0; o < NO; ++o) p[o] = fmaf(S.w3[o * NH + cbase + c], h, p[o]);
        }
#pragma unroll
        for (int o = 0; o < NO; ++o) S.part[warp >> 2][r][o] = p[o];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // Release the accumulator only once the MMAs that write it are known to be complete.
    // After a timeout, wait once more (bounded, 8x as long); if the commit still has not
    // arrived, the columns stay allocated (a late MMA must not write into columns another
    // CTA has been given since) and the error says so.
    bool release = done != 0;
    if (!done) {
        unsigned late = mbar_wait_bounded(mb, 0, 8u * kTcWaitLimit) ? 1u : 0u;
        late = __syncthreads_and(late);
        release = late != 0;
        if (!release && tid == 0) atomicExch(err, 2);
    }
    if (warp == 0 && release) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
    }
    if (!done) return;
    for (int i = tid; i < TILE * NO; i += THREADS) {
        const int r = i / NO, o = i % NO;
        if (r < nvalid) Y[(s0 + r) * NO + o] = S.b3[o] + S.part[0][r][o] + S.part[1][r][o];
    }
}

// ---------------------------------------------------------------------------
// training on the tensor cores.  Per tile of 128 samples the three 64-wide products --
// h1 W2^T (forward), dh2 W2 (the gradient reaching h1) and dh2^T h1 (the gradient of W2)
// -- run as tcgen05 MMAs (M = 128, N = 64, K = 16 per instruction, FP32 accumulators in
// 192 TMEM columns).  The bf16 operands carry the FP32 activations in two parts,
// x = hi + lo with hi = bf16(x) and lo = bf16(x - hi) (about 16 significant bits): W2 is
// bf16 already, so the first two products take hi and lo of the activation (two MMA
// passes), the third hi*hi + hi*lo + lo*hi (three passes; lo*lo is below 2^-16 relative).
// The 6-wide and 3-wide layers, tanh, the loss and the bias gradients stay on the FMA
// pipes as in mlp_tile_kernel, and the tile stores its partial gradient for the same
// fixed-order sum.
// dh2^T h1 is a 64-row product: it is issued with M = 128 and its rows 64..127 (which read
// the operand tiles that follow in shared memory) are not used.
// ---------------------------------------------------------------------------
struct TrainTcSmem {
    alignas(1024) unsigned char wf[NH * NH * 2];       // B, K = 64: W2 [o][k]
    alignas(1024) unsigned char wb[NH * NH * 2];       // B, K = 64: W2^T [k][o]
    alignas(1024) unsigned char a_hi[TILE * NH * 2];   // A, K = 64: h1 [s][k], then dh2 [s][o]
    alignas(1024) unsigned char a_lo[TILE * NH * 2];
    alignas(1024) unsigned char t_hi[NH * TILE * 2];   // A, K = 128: dh2^T [o][s] (64 rows)
    alignas(1024) unsigned char t_lo[NH * TILE * 2];
    alignas(1024) unsigned char h_hi[NH * TILE * 2];   // B, K = 128: h1^T [k][s]
    alignas(1024) unsigned char h_lo[NH * TILE * 2];
    float w1[NH * NI], b1[NH], b2[NH], w3[NO * NH], b3[NO];
    float mean[NI], istd[NI];
    float xn[TILE * NI];
    float h1[TILE * LD];
    float hd[TILE * LD];      // h2, then dh2 (in place), then dh1
    float dy[TILE * NO];
    float red[THREADS / 32];
    alignas(8) unsigned long long mbar;
    unsigned tmem_base;
};

// byte offset of element (row r, k) of a K-major no-swizzle operand of K columns: 8-row x
// 16-byte core matrices, K step 128 B, row-group step K / 8 x 128 B
__device__ __forceinline__ int core_offset_k(int r, int k, int K) {
    return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ unsigned long long smem_desc_sbo(const void* p, unsigned sbo) {
    const unsigned addr = (unsigned)__cvta_generic_to_shared(p);
    unsigned long long d = 0;
    d |= (unsigned long long)((addr >> 4) & 0x3FFF);          // start address
    d |= (unsigned long long)((128 >> 4) & 0x3FFF) << 16;      // leading (K) byte offset
    d |= (unsigned long long)((sbo >> 4) & 0x3FFF) << 32;      // stride (row group) byte offset
    d |= 1ull << 46;                                           // descriptor version (sm_100)
    return d;
}

__device__ __forceinline__ void mma_bf16(unsigned tmem, unsigned long long da,
                                         unsigned long long db, unsigned idesc, unsigned acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// x as hi + lo bf16 parts at byte offsets o_hi / o_lo of the two tiles
__device__ __forceinline__ void put_split(unsigned char* hi, unsigned char* lo, int off, float x) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
    *reinterpret_cast<__nv_bfloat16*>(lo + off) = __float2bfloat16_rn(x - __bfloat162float(h));
}

// 32 consecutive FP32 accumulator columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld32(unsigned taddr, unsigned (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(THREADS)
mlp_train_tc_kernel(const float* __restrict__ wbf, const float* __restrict__ norm,
                    const float* __restrict__ X, const float* __restrict__ Yt, long long B,
                    float* __restrict__ part, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char tt_raw[];
    const unsigned raw_s = (unsigned)__cvta_generic_to_shared(tt_raw);
    TrainTcSmem& S = *reinterpret_cast<TrainTcSmem*>(tt_raw + (((raw_s + 1023u) & ~1023u) - raw_s));
    float* const grad = part + (size_t)blockIdx.x * (NPARAM + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long s0 = (long long)blockIdx.x * TILE;
    const int nvalid = (int)min((long long)TILE, B - s0);

    if (warp == 0) {   // TMEM: 256 columns (D1 at 0, D2 at 64, D3 at 128)
        const unsigned dst = (unsigned)__cvta_generic_to_shared(&S.tmem_base);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(dst));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        const unsigned mb = (unsigned)__cvta_generic_to_shared(&S.mbar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    }
    for (int i = tid; i < NH * NI; i += THREADS) S.w1[i] = wbf[OFF_W1 + i];
    for (int i = tid; i < NH; i += THREADS) {
        S.b1[i] = wbf[OFF_B1 + i];
        S.b2[i] = wbf[OFF_B2 + i];
    }
    for (int i = tid; i < NO * NH; i += THREADS) S.w3[i] = wbf[OFF_W3 + i];
    if (tid < NO) S.b3[tid] = wbf[OFF_B3 + tid];
    if (tid < NI) {
        S.mean[tid] = norm[tid];
        S.istd[tid] = 1.0f / norm[NI + tid];
    }
    for (int i = tid; i < NH * NH; i += THREADS) {
        const int o = i / NH, k = i % NH;
        const __nv_bfloat16 w = __float2bfloat16_rn(wbf[OFF_W2 + i]);   // exact: wbf is bf16
        *reinterpret_cast<__nv_bfloat16*>(S.wf + core_offset_k(o, k, NH)) = w;
        *reinterpret_cast<__nv_bfloat16*>(S.wb + core_offset_k(k, o, NH)) = w;
    }
    __syncthreads();
    for (int i = tid; i < TILE * NI; i += THREADS) {
        const int r = i / NI, f = i % NI;
        S.xn[i] = r < nvalid ? (X[(s0 + r) * NI + f] - S.mean[f]) * S.istd[f] : 0.0f;
    }
    __syncthreads();
    // h1 = tanh(W1 xn + b1): FP32, and split into the two bf16 layouts the MMAs read
    for (int i = tid; i < TILE * NH; i += THREADS) {
        const int r = i / NH, o = i % NH;
        float a = S.b1[o];
#pragma unroll
        for (int f = 0; f < NI; ++f) a = fmaf(S.w1[o * NI + f], S.xn[r * NI + f], a);
        const float h = tanhf(a);
        S.h1[r * LD + o] = h;
        put_split(S.a_hi, S.a_lo, core_offset_k(r, o, NH), h);
        put_split(S.h_hi, S.h_lo, core_offset_k(o, r, TILE), h);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = S.tmem_base;
    const unsigned mb = (unsigned)__cvta_generic_to_shared(&S.mbar);
    const unsigned idesc = mma_idesc();
    if (tid == 0) {   // D1 = (h1_hi + h1_lo) W2^T
        for (int part_i = 0; part_i < 2; ++part_i) {
            const unsigned char* A = part_i ? S.a_lo : S.a_hi;
#pragma unroll
            for (int kk = 0; kk < NH / 16; ++kk)
                mma_bf16(tmem, smem_desc_sbo(A + kk * 256, NH * 16),
                         smem_desc_sbo(S.wf + kk * 256, NH * 16), idesc,
                         (part_i | kk) ? 1u : 0u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(mb) : "memory");
    }
    unsigned done = mbar_wait_bounded(mb, 0, kTcWaitLimit) ? 1u : 0u;
    done = __syncthreads_and(done);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int rbase = 32 * (warp & 3), cbase = 32 * (warp >> 2);
    const unsigned tlane = (unsigned)rbase << 16;
    if (done) {   // h2 = tanh(D1 + b2)
        unsigned v[32];
        tmem_ld32(tmem + tlane + (unsigned)cbase, v);
        const int r = rbase + lane;
#pragma unroll
        for (int c = 0; c < 32; ++c)
            S.hd[r * LD + cbase + c] = tanhf(__uint_as_float(v[c]) + S.b2[cbase + c]);
    }
    __syncthreads();
    // y = W3 h2 + b3, loss, dy
    float lsum = 0.0f;
    for (int i = tid; i < TILE * NO; i += THREADS) {
        const int r = i / NO, o = i % NO;
        float a = S.b3[o];
        for (int k = 0; k < NH; ++k) a = fmaf(S.w3[o * NH + k], S.hd[r * LD + k], a);
        if (r < nvalid) {
            const float d = a - Yt[(s0 + r) * NO + o];
            lsum += d * d;
            S.dy[i] = 2.0f * d / (float)(B * NO);
        } else {
            S.dy[i] = 0.0f;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) S.red[warp] = lsum;
    __syncthreads();
    if (tid == 0) {
        float t = 0.0f;
        for (int w = 0; w < THREADS / 32; ++w) t += S.red[w];
        grad[NPARAM] = t / (float)(B * NO);
    }
    // dW3, db3
    if (tid < NO * NH) {
        const int o = tid / NH, k = tid % NH;
        float g = 0.0f;
        for (int r = 0; r < TILE; ++r) g = fmaf(S.dy[r * NO + o], S.hd[r * LD + k], g);
        grad[OFF_W3 + tid] = g;
    } else if (tid < NO * NH + NO) {
        const int o = tid - NO * NH;
        float g = 0.0f;
        for (int r = 0; r < TILE; ++r) g += S.dy[r * NO + o];
        grad[OFF_B3 + o] = g;
    }
    __syncthreads();
    // dh2 = (W3^T dy) (1 - h2^2), in place, and split into the layouts of the backward MMAs
    for (int i = tid; i < TILE * NH; i += THREADS) {
        const int r = i / NH, k = i % NH;
        float a = 0.0f;
#pragma unroll
        for (int o = 0; o < NO; ++o) a = fmaf(S.dy[r * NO + o], S.w3[o * NH + k], a);
        const float h = S.hd[r * LD + k];
        const float d = a * (1.0f - h * h);
        S.hd[r * LD + k] = d;
        put_split(S.a_hi, S.a_lo, core_offset_k(r, k, NH), d);
        put_split(S.t_hi, S.t_lo, core_offset_k(k, r, TILE), d);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0 && done) {
        // D2 = (dh2_hi + dh2_lo) W2
        for (int part_i = 0; part_i < 2; ++part_i) {
            const unsigned char* A = part_i ? S.a_lo : S.a_hi;
#pragma unroll
            for (int kk = 0; kk < NH / 16; ++kk)
                mma_bf16(tmem + 64, smem_desc_sbo(A + kk * 256, NH * 16),
                         smem_desc_sbo(S.wb + kk * 256, NH * 16), idesc,
                         (part_i | kk) ? 1u : 0u);
        }
        // D3 = dh2^T h1 over the 128 samples: hi hi + hi lo + lo hi
        for (int part_i = 0; part_i < 3; ++part_i) {
            const unsigned char* A = part_i == 2 ? S.t_lo : S.t_hi;
            const unsigned char* Bm = part_i == 1 ? S.h_lo : S.h_hi;
#pragma unroll
            for (int kk = 0; kk < TILE / 16; ++kk)
                mma_bf16(tmem + 128, smem_desc_sbo(A + kk * 256, TILE * 16),
                         smem_desc_sbo(Bm + kk * 256, TILE * 16), idesc,
                         (part_i | kk) ? 1u : 0u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(mb) : "memory");
    }
    // db2 while the MMAs run
    if (tid < NH) {
        float gb = 0.0f;
        for (int r = 0; r < TILE; ++r) gb += S.hd[r * LD + tid];
        grad[OFF_B2 + tid] = gb;
    }
    unsigned done2 = done ? (mbar_wait_bounded(mb, 1, kTcWaitLimit) ? 1u : 0u) : 0u;
    done2 = __syncthreads_and(done2);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (done2) {
        unsigned v[32];
        // dh1 = D2 (1 - h1^2), over dh2 (db2 has been summed above)
        tmem_ld32(tmem + tlane + 64u + (unsigned)cbase, v);
        const int r = rbase + lane;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const float h = S.h1[r * LD + cbase + c];
            S.hd[r * LD + cbase + c] = __uint_as_float(v[c]) * (1.0f - h * h);
        }
        // dW2 [o][k]: rows 0..63 of D3 (warps 0, 1, 4, 5 hold them)
        if (rbase < NH) {
            tmem_ld32(tmem + tlane + 128u + (unsigned)cbase, v);
            float* g = grad + OFF_W2 + (size_t)r * NH + cbase;
#pragma unroll
            for (int c = 0; c < 32; c += 4)
                *reinterpret_cast<float4*>(g + c) =
                    make_float4(__uint_as_float(v[c]), __uint_as_float(v[c + 1]),
                                __uint_as_float(v[c + 2]), __uint_as_float(v[c + 3]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // Release the accumulators only once the MMAs writing them are known to be complete
    // (as in mlp_forward_tc_kernel); a tile whose waits ran out stores a zero gradient.
    bool release = done2 != 0;
    if (!done2) {
        const unsigned phase = done ? 1u : 0u;
        unsigned late = mbar_wait_bounded(mb, phase, 8u * kTcWaitLimit) ? 1u : 0u;
        late = __syncthreads_and(late);
        release = late != 0;
        if (tid == 0) atomicExch(err, release ? 1 : 2);
        for (int i = tid; i <= NPARAM; i += THREADS) grad[i] = 0.0f;
    }
    if (warp == 0 && release) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
    }
    if (!done2) return;
    __syncthreads();
    // dW1[o][f] = sum_s dh1[s][o] xn[s][f]; db1
    for (int i = tid; i < NH * NI + NH; i += THREADS) {
        if (i < NH * NI) {
            const int o = i / NI, f = i % NI;
            float g = 0.0f;
            for (int r = 0; r < TILE; ++r) g = fmaf(S.hd[r * LD + o], S.xn[r * NI + f], g);
            grad[OFF_W1 + i] = g;
        } else {
            const int o = i - NH * NI;
            float g = 0.0f;
            for (int r = 0; r < TILE; ++r) g += S.hd[r * LD + o];
            grad[OFF_B1 + o] = g;
        }
    }
}

// Adam (Kingma & Ba 2015) on the FP32 master weights; also refreshes the bf16-rounded copy.
// grad[i] = sum over tiles t of part[t][i], t ascending (i = NPARAM: the loss)
__global__ void grad_sum_kernel(const float* __restrict__ part, long long tiles,
                                float* __restrict__ grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > NPARAM) return;
    float g = 0.0f;
    for (long long t = 0; t < tiles; ++t) g += part[(size_t)t * (NPARAM + 1) + i];
    grad[i] = g;
}

__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ wbf,
                            float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float lr, float b1, float b2, float c1,
                            float c2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float t = theta[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    theta[i] = t;
    wbf[i] = __bfloat162float(__float2bfloat16_rn(t));
}

__global__ void round_bf16_kernel(const float* __restrict__ theta, float* __restrict__ wbf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NPARAM) wbf[i] = __bfloat162float(__float2bfloat16_rn(theta[i]));
}

// splitmix64 (Steele, Lea & Flood 2014) as a counter-based generator for minibatch rows.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void gather_kernel(const float* __restrict__ X, const float* __restrict__ Yt, long long N,
                              int batch, unsigned long long key, float* __restrict__ Xb,
                              float* __restrict__ Yb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch) return;
    const long long r = (long long)(splitmix64(key + (unsigned long long)i) % (unsigned long long)N);
#pragma unroll
    for (int f = 0; f < NI; ++f) Xb[i * NI + f] = X[r * NI + f];
#pragma unroll
    for (int o = 0; o < NO; ++o) Yb[i * NO + o] = Yt[r * NO + o];
}

// per-feature sum and sum of squares (FP64) for the input standardisation
__global__ void moments_kernel(const float* __restrict__ X, long long N, double* __restrict__ acc) {
    double s[NI] = {}, q[NI] = {};
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x)
#pragma unroll
        for (int f = 0; f < NI; ++f) {
            const double x = X[r * NI + f];
            s[f] += x;
            q[f] += x * x;
        }
#pragma unroll
    for (int f = 0; f < NI; ++f) {
        atomicAdd(acc + f, s[f]);
        atomicAdd(acc + NI + f, q[f]);
    }
}

__global__ void finish_moments_kernel(const double* __restrict__ acc, long long N,
                                      float* __restrict__ norm) {
    const int f = threadIdx.x;
    if (f >= NI) return;
    const double mean = acc[f] / (double)N;
    const double var = fmax(acc[NI + f] / (double)N - mean * mean, 0.0);
    norm[f] = (float)mean;
    norm[NI + f] = (float)fmax(sqrt(var), 1e-6);
}

}  // namespace

struct rc_mlp_s {
    int device = 0;
    float* d = nullptr;   // theta | wbf | m | v | grad | norm(2 NI) | loss | gather buffers
    float *theta, *wbf, *m, *v, *grad, *norm, *loss;
    double* d_mom = nullptr;
    float* Xb = nullptr;
    float* Yb = nullptr;
    int batch_cap = 0;
    float* Ysc = nullptr;          // forward scratch for seeding
    long long ysc_cap = 0;
    long long step = 0;
    unsigned long long seed = 0;
    float* h_loss = nullptr;       // pinned
    bool tensor_cores = false;     // inference through mlp_forward_tc_kernel
    bool tc_train = false;         // loss and gradient through mlp_train_tc_kernel
    int* d_err = nullptr;          // set if a tensor-core wait ran out
    float* part = nullptr;         // per-tile partial gradients and losses [tiles][NPARAM + 1]
    long long part_tiles = 0;
};

namespace {

size_t smem_bytes() { return sizeof(Smem); }
size_t tc_smem_bytes() { return sizeof(TcSmem) + 1024; }   // + alignment slack
size_t tt_smem_bytes() { return sizeof(TrainTcSmem) + 1024; }

rc_status ensure_configured() {
    static bool done = false;
    if (done) return RC_OK;
    cudaError_t e = cudaFuncSetAttribute(mlp_tile_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_tile_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tc_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tt_smem_bytes());
    if (e != cudaSuccess) return mcuda(e, "mlp: shared-memory opt-in");
    done = true;
    return RC_OK;
}

rc_status loss_grad(rc_mlp_t n, const float* X, const float* Yt, long long B, cudaStream_t s) {
    rc_status st = ensure_configured();
    if (st != RC_OK) return st;
    const long long tiles = (B + TILE - 1) / TILE;
    cudaError_t e;
    if (n->part_tiles < tiles) {
        cudaStreamSynchronize(s);
        cudaFree(n->part);
        n->part = nullptr;
        n->part_tiles = 0;
        if ((e = cudaMalloc(&n->part, (size_t)tiles * (NPARAM + 1) * sizeof(float))) != cudaSuccess)
            return mcuda(e, "mlp: partial-gradient buffer");
        n->part_tiles = tiles;
    }
    if (n->tc_train)
        mlp_train_tc_kernel<<<(unsigned)tiles, THREADS, tt_smem_bytes(), s>>>(n->wbf, n->norm, X, Yt,
                                                                             B, n->part, n->d_err);
    else
        mlp_tile_kernel<true><<<(unsigned)tiles, THREADS, smem_bytes(), s>>>(n->wbf, n->norm, X, Yt,
                                                                            B, nullptr, n->part);
    // grad and the loss after it: the tiles' partials summed in tile order
    grad_sum_kernel<<<(NPARAM + 1 + 255) / 256, 256, 0, s>>>(n->part, tiles, n->grad);
    e = cudaGetLastError();
    return e == cudaSuccess ? RC_OK : mcuda(e, "mlp_tile_kernel");
}

}  // namespace

extern "C" {

rc_status rc_mlp_create(unsigned long long seed, rc_mlp_t* out) {
    rcx::set_last_error("");
    if (!out) return mfail(RC_ERR_ARG, "rc_mlp_create: out is NULL");
    *out = nullptr;
    rc_mlp_s* n = new (std::nothrow) rc_mlp_s();
    if (!n) return mfail(RC_ERR_OOM, "rc_mlp_create: host allocation");
    cudaGetDevice(&n->device);
    n->seed = seed;
    const size_t floats = 5 * (size_t)NPARAM + 2 * NI + 4;
    cudaError_t e = cudaMalloc(&n->d, floats * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->d_mom, 2 * NI * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&n->h_loss, sizeof(float));
    if (e != cudaSuccess) {
        cudaFree(n->d);
        cudaFree(n->d_mom);
        delete n;
        return mcuda(e, "rc_mlp_create");
    }
    n->theta = n->d;
    n->wbf = n->theta + NPARAM;
    n->m = n->wbf + NPARAM;
    n->v = n->m + NPARAM;
    n->grad = n->v + NPARAM;
    n->loss = n->grad + NPARAM;      // right after grad: one memset clears both
    n->norm = n->loss + 4;
    // Glorot-uniform weights, zero biases, identity standardisation
    std::vector<float> h(floats, 0.0f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int off, int fan_out, int fan_in) {
        const double a = std::sqrt(6.0 / (fan_in + fan_out));
        std::uniform_real_distribution<double> U(-a, a);
        for (int i = 0; i < fan_out * fan_in; ++i) h[off + i] = (float)U(rng);
    };
    fill(OFF_W1, NH, NI);
    fill(OFF_W2, NH, NH);
    fill(OFF_W3, NO, NH);
    for (int f = 0; f < NI; ++f) h[5 * NPARAM + 4 + NI + f] = 1.0f;
    e = cudaMemcpy(n->d, h.data(), floats * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        round_bf16_kernel<<<(NPARAM + 255) / 256, 256>>>(n->theta, n->wbf);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        cudaFree(n->d);
        cudaFree(n->d_mom);
        cudaFreeHost(n->h_loss);
        delete n;
        return mcuda(e, "rc_mlp_create: upload");
    }
    *out = n;
    return RC_OK;
}

void rc_mlp_destroy(rc_mlp_t n) {
    if (!n) return;
    cudaDeviceSynchronize();
    cudaFree(n->d);
    cudaFree(n->d_mom);
    cudaFree(n->Xb);
    cudaFree(n->Ysc);
    cudaFree(n->d_err);
    cudaFree(n->part);
    cudaFreeHost(n->h_loss);
    delete n;
}

int rc_mlp_n_params(rc_mlp_t n) { return n ? NPARAM : 0; }

rc_status rc_mlp_set_params(rc_mlp_t n, const float* theta, const float* mean, const float* std_) {
    rcx::set_last_error("");
    if (!n) return mfail(RC_ERR_ARG, "rc_mlp_set_params: NULL network");
    cudaError_t e = cudaSuccess;
    if (theta) e = cudaMemcpy(n->theta, theta, NPARAM * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && mean) e = cudaMemcpy(n->norm, mean, NI * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && std_) e = cudaMemcpy(n->norm + NI, std_, NI * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && theta) {
        round_bf16_kernel<<<(NPARAM + 255) / 256, 256>>>(n->theta, n->wbf);
        cudaMemset(n->m, 0, 2 * NPARAM * sizeof(float));
        n->step = 0;
        e = cudaDeviceSynchronize();
    }
    return e == cudaSuccess ? RC_OK : mcuda(e, "rc_mlp_set_params");
}

rc_status rc_mlp_get_params(rc_mlp_t n, float* theta, float* mean, float* std_) {
    rcx::set_last_error("");
    if (!n) return mfail(RC_ERR_ARG, "rc_mlp_get_params: NULL network");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && theta) e = cudaMemcpy(theta, n->theta, NPARAM * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && mean) e = cudaMemcpy(mean, n->norm, NI * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && std_) e = cudaMemcpy(std_, n->norm + NI, NI * sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? RC_OK : mcuda(e, "rc_mlp_get_params");
}

rc_status rc_mlp_fit_normalization(rc_mlp_t n, const float* X, long long N, void* stream) {
    rcx::set_last_error("");
    if (!n || !X || N < 1) return mfail(RC_ERR_ARG, "rc_mlp_fit_normalization: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(n->d_mom, 0, 2 * NI * sizeof(double), s);
    moments_kernel<<<256, 256, 0, s>>>(X, N, n->d_mom);
    finish_moments_kernel<<<1, 32, 0, s>>>(n->d_mom, N, n->norm);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RC_OK : mcuda(e, "rc_mlp_fit_normalization");
}

rc_status rc_mlp_forward(rc_mlp_t n, const float* X, long long B, float* Y, void* stream) {
    rcx::set_last_error("");
    if (!n || !X || !Y || B < 0) return mfail(RC_ERR_ARG, "rc_mlp_forward: bad arguments");
    if (B == 0) return RC_OK;
    rc_status st = ensure_configured();
    if (st != RC_OK) return st;
    if (n->tensor_cores) {
        mlp_forward_tc_kernel<<<(unsigned)((B + TILE - 1) / TILE), THREADS, tc_smem_bytes(),
                                (cudaStream_t)stream>>>(n->wbf, n->norm, X, B, Y, n->d_err);
    } else {
        mlp_tile_kernel<false><<<(unsigned)((B + TILE - 1) / TILE), THREADS, smem_bytes(),
                                 (cudaStream_t)stream>>>(n->wbf, n->norm, X, nullptr, B, Y, nullptr);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RC_OK : mcuda(e, "rc_mlp_forward");
}

rc_status rc_mlp_use_tensor_cores(rc_mlp_t n, int enable) {
    rcx::set_last_error("");
    if (!n) return mfail(RC_ERR_ARG, "rc_mlp_use_tensor_cores: NULL network");
    if (enable && !n->d_err) {
        cudaError_t e = cudaMalloc(&n->d_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(n->d_err, 0, sizeof(int));
        if (e != cudaSuccess) return mcuda(e, "rc_mlp_use_tensor_cores");
    }
    n->tensor_cores = (enable & RC_MLP_TC_INFERENCE) != 0;
    n->tc_train = (enable & RC_MLP_TC_TRAINING) != 0;
    return RC_OK;
}

rc_status rc_surrogate_init(unsigned long long seed, rc_mlp_t* out) { return rc_mlp_create(seed, out); }

rc_status rc_surrogate_train_step(rc_mlp_t net, const float* X, const float* Y_target, long long N,
                                  int batch, float lr, float* loss, void* stream) {
    return rc_mlp_train(net, X, Y_target, N, batch, 1, lr, loss, stream);
}

rc_status rc_surrogate_predict(rc_mlp_t net, const float* X, long long B, float* Y, void* stream) {
    return rc_mlp_forward(net, X, B, Y, stream);
}

rc_status rc_selftest_bounded_wait(void* stream) {
    rcx::set_last_error("");
    cudaStream_t s = (cudaStream_t)stream;
    int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int));
    if (e != cudaSuccess) return mcuda(e, "rc_selftest_bounded_wait");
    int h = -1;
    if ((e = cudaMemsetAsync(d, 0xff, sizeof(int), s)) == cudaSuccess) {
        wait_timeout_probe_kernel<<<1, 32, 0, s>>>(1u << 12, d);   // ~0.3 ms of polling
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return mcuda(e, "rc_selftest_bounded_wait");
    if (h == 1) return mfail(RC_ERR_TIMEOUT, "bounded device wait gave up (as the self-test expects)");
    return mfail(RC_ERR_CUDA, "rc_selftest_bounded_wait: the probe's wait did not give up");
}

rc_status rc_mlp_tensor_core_status(rc_mlp_t n) {
    rcx::set_last_error("");
    if (!n) return mfail(RC_ERR_ARG, "rc_mlp_tensor_core_status: NULL network");
    if (!n->d_err) return RC_OK;
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, n->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return mcuda(e, "rc_mlp_tensor_core_status");
    if (h == 2)
        return mfail(RC_ERR_TIMEOUT, "tensor-core MMA wait ran out and the MMAs never completed: "
                                     "their tensor-memory columns were left allocated");
    return h ? mfail(RC_ERR_TIMEOUT, "tensor-core MMA wait ran out") : RC_OK;
}

rc_status rc_mlp_loss_grad(rc_mlp_t n, const float* X, const float* Yt, long long B, float* grad,
                           float* loss, void* stream) {
    rcx::set_last_error("");
    if (!n || !X || !Yt || B < 1) return mfail(RC_ERR_ARG, "rc_mlp_loss_grad: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    rc_status st = loss_grad(n, X, Yt, B, s);
    if (st != RC_OK) return st;
    cudaError_t e = cudaSuccess;
    if (grad) e = cudaMemcpyAsync(grad, n->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? RC_OK : mcuda(e, "rc_mlp_loss_grad");
}

rc_status rc_mlp_train(rc_mlp_t n, const float* X, const float* Yt, long long N, int batch,
                       int steps, float lr, float* loss_history, void* stream) {
    rcx::set_last_error("");
    if (!n || !X || !Yt || N < 1 || batch < 1 || steps < 0 || !(lr > 0))
        return mfail(RC_ERR_ARG, "rc_mlp_train: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (n->batch_cap < batch) {
        cudaStreamSynchronize(s);
        cudaFree(n->Xb);
        n->Xb = n->Yb = nullptr;
        n->batch_cap = 0;
        if ((e = cudaMalloc(&n->Xb, (size_t)batch * (NI + NO) * sizeof(float))) != cudaSuccess)
            return mcuda(e, "rc_mlp_train: minibatch buffers");
        n->Yb = n->Xb + (size_t)batch * NI;
        n->batch_cap = batch;
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int it = 0; it < steps; ++it) {
        ++n->step;
        const unsigned long long key = n->seed * 0x100000001B3ULL + ((unsigned long long)n->step << 32);
        gather_kernel<<<(batch + 255) / 256, 256, 0, s>>>(X, Yt, N, batch, key, n->Xb, n->Yb);
        rc_status st = loss_grad(n, n->Xb, n->Yb, batch, s);
        if (st != RC_OK) return st;
        const double c1 = 1.0 / (1.0 - std::pow((double)b1, (double)n->step));
        const double c2 = 1.0 / (1.0 - std::pow((double)b2, (double)n->step));
        adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(n->theta, n->wbf, n->m, n->v, n->grad, lr,
                                                         b1, b2, (float)c1, (float)c2, eps);
        if (loss_history) {
            cudaMemcpyAsync(n->h_loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return mcuda(e, "rc_mlp_train");
            loss_history[it] = *n->h_loss;
        }
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? RC_OK : mcuda(e, "rc_mlp_train");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// features, targets and the seed of the non-LTE iteration (need the atom's tables)
// ---------------------------------------------------------------------------
namespace {

__global__ void features_kernel(const double* __restrict__ T, const double* __restrict__ ne,
                                const double* __restrict__ nH, const float* __restrict__ J,
                                long long ncell, int l0, int l1, int l2, float* __restrict__ X) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    float* x = X + c * NI;
    x[0] = (float)log10(T[c]);
    x[1] = (float)log10(fmax(ne[c], 1e-300));
    x[2] = (float)log10(fmax(nH[c], 1e-300));
    const int ls[3] = {l0, l1, l2};
#pragma unroll
    for (int l = 0; l < 3; ++l) x[3 + l] = log10f(fmaxf(J[(size_t)ls[l] * ncell + c], 1e-38f));
}

__global__ void targets_kernel(const double* __restrict__ T, const double* __restrict__ n_atom,
                               const double* __restrict__ pops, const double* __restrict__ Ek,
                               const double* __restrict__ g, int nlev, long long ncell,
                               float* __restrict__ Y) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    double b[8], sum = 0.0;
    for (int i = 0; i < nlev; ++i) {
        b[i] = g[i] * exp(-Ek[i] / T[c]);
        sum += b[i];
    }
    for (int i = 0; i < nlev && i < NO; ++i) {
        const double lte = n_atom[c] * b[i] / sum;
        Y[c * NO + i] = (float)log10(pops[(size_t)i * ncell + c] / lte);
    }
}

__global__ void seed_kernel(const float* __restrict__ Y, const double* __restrict__ T,
                            const double* __restrict__ n_atom, const double* __restrict__ Ek,
                            const double* __restrict__ g, int nlev, long long ncell,
                            double* __restrict__ pops, int* __restrict__ n_fallback) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    double lte[8], sum = 0.0;
    for (int i = 0; i < nlev; ++i) {
        lte[i] = g[i] * exp(-Ek[i] / T[c]);
        sum += lte[i];
    }
    double p[8], tot = 0.0;
    bool ok = true;
    for (int i = 0; i < nlev; ++i) {
        lte[i] *= n_atom[c] / sum;
        const double y = i < NO ? (double)Y[c * NO + i] : 0.0;
        p[i] = lte[i] * exp10(fmin(fmax(y, -30.0), 30.0));
        ok = ok && isfinite(y) && p[i] > 0.0;
        tot += p[i];
    }
    // the LTE start is the fallback wherever the network's output is unusable
    if (!ok || !(tot > 0.0) || !isfinite(tot)) {
        atomicAdd(n_fallback, 1);
        for (int i = 0; i < nlev; ++i) pops[(size_t)i * ncell + c] = lte[i];
        return;
    }
    for (int i = 0; i < nlev; ++i) pops[(size_t)i * ncell + c] = p[i] * n_atom[c] / tot;
}

}  // namespace

extern "C" {

rc_status rc_surrogate_features(rc_atom_t atom, const double* T, const double* ne, const double* nH,
                                const float* J, long long ncell, float* X, void* stream) {
    rcx::set_last_error("");
    if (!atom || !T || !ne || !nH || !J || !X || ncell < 0)
        return mfail(RC_ERR_ARG, "rc_surrogate_features: bad arguments");
    const double *Ek, *g;
    int nlev, npl, nlines;
    rc_status st = rcx::atom_levels(atom, &Ek, &g, &nlev, &npl, &nlines);
    if (st != RC_OK) return st;
    if (nlines < 3) return mfail(RC_ERR_UNSUPPORTED, "rc_surrogate_features: needs 3 lines");
    if (ncell == 0) return RC_OK;
    features_kernel<<<(unsigned)((ncell + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        T, ne, nH, J, ncell, npl / 2, npl + npl / 2, 2 * npl + npl / 2, X);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RC_OK : mcuda(e, "rc_surrogate_features");
}

rc_status rc_surrogate_targets(rc_atom_t atom, const double* T, const double* n_atom,
                               const double* pops, long long ncell, float* Y, void* stream) {
    rcx::set_last_error("");
    if (!atom || !T || !n_atom || !pops || !Y || ncell < 0)
        return mfail(RC_ERR_ARG, "rc_surrogate_targets: bad arguments");
    const double *Ek, *g;
    int nlev, npl, nlines;
    rc_status st = rcx::atom_levels(atom, &Ek, &g, &nlev, &npl, &nlines);
    if (st != RC_OK) return st;
    if (nlev != NO) return mfail(RC_ERR_UNSUPPORTED, "rc_surrogate_targets: the network predicts 3 levels");
    if (ncell == 0) return RC_OK;
    targets_kernel<<<(unsigned)((ncell + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        T, n_atom, pops, Ek, g, nlev, ncell, Y);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RC_OK : mcuda(e, "rc_surrogate_targets");
}

rc_status rc_surrogate_seed(rc_atom_t atom, rc_mlp_t net, const float* X, const double* T,
                            const double* n_atom, long long ncell, double* pops, int* n_fallback,
                            void* stream) {
    rcx::set_last_error("");
    if (!atom || !net || !X || !T || !n_atom || !pops || ncell < 0)
        return mfail(RC_ERR_ARG, "rc_surrogate_seed: bad arguments");
    const double *Ek, *g;
    int nlev, npl, nlines;
    rc_status st = rcx::atom_levels(atom, &Ek, &g, &nlev, &npl, &nlines);
    if (st != RC_OK) return st;
    if (nlev != NO) return mfail(RC_ERR_UNSUPPORTED, "rc_surrogate_seed: the network predicts 3 levels");
    if (ncell == 0) return RC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (net->ysc_cap < ncell) {
        cudaStreamSynchronize(s);
        cudaFree(net->Ysc);
        net->Ysc = nullptr;
        net->ysc_cap = 0;
        if ((e = cudaMalloc(&net->Ysc, (size_t)ncell * NO * sizeof(float) + 16)) != cudaSuccess)
            return mcuda(e, "rc_surrogate_seed: scratch");
        net->ysc_cap = ncell;
    }
    int* d_fb = reinterpret_cast<int*>(net->Ysc + (size_t)ncell * NO);
    cudaMemsetAsync(d_fb, 0, sizeof(int), s);
    st = rc_mlp_forward(net, X, ncell, net->Ysc, stream);
    if (st != RC_OK) return st;
    seed_kernel<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(net->Ysc, T, n_atom, Ek, g, nlev,
                                                                ncell, pops, d_fb);
    if ((e = cudaGetLastError()) != cudaSuccess) return mcuda(e, "rc_surrogate_seed");
    if (n_fallback) {
        if ((e = cudaMemcpyAsync(n_fallback, d_fb, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return mcuda(e, "rc_surrogate_seed: fallback count");
    }
    return RC_OK;
}

}  // extern "C"
