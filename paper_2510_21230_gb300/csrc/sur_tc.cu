// sur_tc.cu -- the surrogate MLP (32 -> 64 -> 64 -> 3, SiLU) on the
// fifth-generation tensor cores: tcgen05.mma with bfloat16 operands staged in
// shared memory and FP32 accumulators in tensor memory (TMEM).
//
// A persistent CTA of 128 threads takes 128-row tiles.  The input tile (stored
// by the descriptor kernel already in the operand layout) arrives by a bulk
// asynchronous copy (cp.async.bulk on the TMA engine) issued one tile ahead,
// completing on an mbarrier; each thread reads its row's 16 vectors from
// global memory (L2, where the descriptor kernel left them) in the epilogue.  Thread t owns row t: after each
// layer it reads
// the row's accumulators back from TMEM lane t (tcgen05.ld 32x32b), applies
// bias + SiLU and writes the next layer's operand row -- no shuffles, no
// shared-memory transposes.  (Raw FP32 input rows are normalised and staged by
// the threads instead.)  One elected thread issues the MMAs (M = 128,
// N = 64 / 64 / 16, K = 16 per instruction) and commits them to an mbarrier
// that all threads wait on with a bounded number of tries.
//
// Operands use the canonical K-major layout without swizzle: 8-row x 16-byte
// core matrices, core matrix (row group g, 8-element chunk j) at byte
// g * SBO + j * LBO with LBO = 128 and SBO = (K / 8) * 128.  TMEM columns:
// layer 1 in [0, 64), layer 2 in [64, 128), layer 3 in [0, 16) (layer 1 is
// consumed by then); 128 columns per CTA.
#include <cuda_bf16.h>
#include <stdint.h>

#include "surrogate.cuh"
#include "tc_common.cuh"

namespace atm3 {

namespace {
using namespace tc;

constexpr int TC_M = 128;           // rows per tile = TMEM lanes
constexpr uint32_t TC_COLS = 128;   // TMEM columns per CTA

static_assert(TC_M == SUR_TILE_M && TC_LBO == 128, "the tile layout is the operand layout");

struct TcSmem {
    alignas(128) unsigned char w1[64 * 32 * 2];   // W1^T  N 64 x K 32
    alignas(128) unsigned char w2[64 * 64 * 2];   // W2^T  N 64 x K 64
    alignas(128) unsigned char w3[16 * 64 * 2];   // W3^T  N 16 x K 64
    alignas(128) unsigned char x[TC_M * 32 * 2];  // input tile   M 128 x K 32
    alignas(128) unsigned char h[TC_M * 64 * 2];  // hidden tile  M 128 x K 64
    float b1[64], b2[64], b3[16];
    alignas(8) unsigned long long mbar;           // MMA completion
    alignas(8) unsigned long long xbar;           // bulk-copy completion
    uint32_t tmem_base;
};

constexpr uint32_t TC_X_BYTES = TC_M * 32 * 2;

template <bool BF16_IN>
__global__ void __launch_bounds__(TC_M) k_sur_mlp_tc(long long n, const float* __restrict__ Din,
                                                     const __nv_bfloat16* __restrict__ Xin,
                                                     const float* __restrict__ Vin,
                                                     const SurPacked* __restrict__ model, float* w,
                                                     float* f, double* f_soa, int* status)
{
    __shared__ TcSmem S;
    const int tid = threadIdx.x, warp = tid >> 5;

    // weights in the canonical layouts (16-byte chunks of the packed rows)
    for (int e = tid; e < 64 * 4; e += TC_M) {
        const int r = e >> 2, j = e & 3;
        put_chunk(S.w1, r, j, 4, *reinterpret_cast<const uint4*>(model->w1t + r * SUR_XS + 8 * j));
    }
    for (int e = tid; e < 64 * 8; e += TC_M) {
        const int r = e >> 3, j = e & 7;
        put_chunk(S.w2, r, j, 8, *reinterpret_cast<const uint4*>(model->w2t + r * SUR_HS + 8 * j));
    }
    for (int e = tid; e < 16 * 8; e += TC_M) {
        const int r = e >> 3, j = e & 7;
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        put_chunk(S.w3, r, j, 8, r < SUR_NO ? *reinterpret_cast<const uint4*>(model->w3t + r * SUR_HS + 8 * j) : z);
    }
    if (tid < 64) {
        S.b1[tid] = model->b1[tid];
        S.b2[tid] = model->b2[tid];
    }
    if (tid < 16) S.b3[tid] = tid < SUR_NO ? model->b3[tid] : 0.0f;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.xbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&S.tmem_base)),
                     "r"(TC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;  // this warp's TMEM lane quarter
    const uint32_t id64 = idesc_bf16(TC_M, 64), id16 = idesc_bf16(TC_M, 16);

    uint32_t phase = 0u, xphase = 0u;
    bool ok = true;
    // every thread waits on a barrier phase; all agree on the outcome
    auto wait_bar = [&](unsigned long long* bar, uint32_t& ph) {
        bool done = false;
        for (long it = 0; it < TC_WAIT_TRIES && !done; it++) done = mbar_try_wait(bar, ph);
        ph ^= 1u;
        ok = __syncthreads_and(done) != 0;
    };
    auto wait_mma = [&]() {
        wait_bar(&S.mbar, phase);
        tc_fence_after();
    };
    // the next tile's inputs: one bulk copy of the X tile
    auto prefetch = [&](long long tile) {
        if (tid == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&S.xbar)),
                         "r"(TC_X_BYTES)
                         : "memory");
            bulk_g2s(S.x, Xin + tile * (TC_M * SUR_ND), TC_X_BYTES, &S.xbar);
        }
    };
    // bias + SiLU of 64 accumulator columns at TMEM column c0, written as row
    // `tid` of the hidden operand
    auto hidden = [&](uint32_t c0, const float* bias) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            float v[16];
            tmem_ld16(tmem + lane_base + c0 + 16 * q, v);
            uint32_t p[8];
#pragma unroll
            for (int i = 0; i < 8; i++)
                p[i] = pack_bf2(silu(v[2 * i] + bias[16 * q + 2 * i]), silu(v[2 * i + 1] + bias[16 * q + 2 * i + 1]));
            put_chunk(S.h, tid, 2 * q, 8, make_uint4(p[0], p[1], p[2], p[3]));
            put_chunk(S.h, tid, 2 * q + 1, 8, make_uint4(p[4], p[5], p[6], p[7]));
        }
        tc_fence_before();
        fence_async_smem();
        __syncthreads();
    };

    const long long ntiles = (n + TC_M - 1) / TC_M;
    if (BF16_IN && blockIdx.x < ntiles) prefetch(blockIdx.x);
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long s = tile * TC_M + tid;
        const bool active = s < n;
        if (BF16_IN) {
            wait_bar(&S.xbar, xphase);
            if (!ok) break;
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                uint32_t p[4];
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int k = 8 * j + 2 * i;
                    const float a = active ? (Din[s * SUR_ND + k] - model->mean[k]) / model->scale[k] : 0.0f;
                    const float b = active ? (Din[s * SUR_ND + k + 1] - model->mean[k + 1]) / model->scale[k + 1] : 0.0f;
                    p[i] = pack_bf2(a, b);
                }
                put_chunk(S.x, tid, j, 4, make_uint4(p[0], p[1], p[2], p[3]));
            }
            fence_async_smem();
            __syncthreads();
        }

        // layer 1: TMEM [0, 64) = X W1
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < 2; kk++)
                umma_bf16(tmem, sdesc(S.x + kk * 2 * TC_LBO, 4 * 128), sdesc(S.w1 + kk * 2 * TC_LBO, 4 * 128),
                          id64, kk > 0);
            umma_commit(&S.mbar);
        }
        wait_mma();
        if (!ok) break;
        // the X tile is consumed: fetch the next tile's meanwhile
        if (BF16_IN && tile + gridDim.x < ntiles) prefetch(tile + gridDim.x);
        hidden(0u, S.b1);

        // layer 2: TMEM [64, 128) = H1 W2
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < 4; kk++)
                umma_bf16(tmem + 64u, sdesc(S.h + kk * 2 * TC_LBO, 8 * 128), sdesc(S.w2 + kk * 2 * TC_LBO, 8 * 128),
                          id64, kk > 0);
            umma_commit(&S.mbar);
        }
        wait_mma();
        if (!ok) break;
        hidden(64u, S.b2);

        // layer 3: TMEM [0, 16) = H2 W3 (layer 1's columns are consumed)
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < 4; kk++)
                umma_bf16(tmem, sdesc(S.h + kk * 2 * TC_LBO, 8 * 128), sdesc(S.w3 + kk * 2 * TC_LBO, 8 * 128),
                          id16, kk > 0);
            umma_commit(&S.mbar);
        }
        wait_mma();
        if (!ok) break;
        float o[16];
        tmem_ld16(tmem + lane_base, o);
        if (active) {
            float wm[SUR_NO];
#pragma unroll
            for (int m = 0; m < SUR_NO; m++) {
                wm[m] = o[m] + S.b3[m];
                if (w) w[s * SUR_NO + m] = wm[m];
            }
            const float* vrow = Vin + s * SUR_NV;
            float fc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int m = 0; m < SUR_NO; m++)
#pragma unroll
                for (int c = 0; c < 3; c++) fc[c] = fmaf(wm[m], vrow[3 * m + c], fc[c]);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                if (f) f[s * 3 + c] = fc[c];
                if (f_soa) f_soa[c * n + s] = (double)fc[c];
            }
        }
        tc_fence_before();
        __syncthreads();  // TMEM read and operands consumed before the next tile overwrites them
        tc_fence_after();
    }
    // a bulk copy still in flight (a wait gave up) lands before shared memory is released
    if (BF16_IN && !ok) {
        bool done = false;
        for (long it = 0; it < TC_WAIT_TRIES && !done; it++) done = mbar_try_wait(&S.xbar, xphase);
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS)
                     : "memory");
    if (!ok && tid == 0) atomicOr(status, ST_TIMEOUT);
}

}  // namespace

cudaError_t launch_sur_mlp_tc(long long n, const float* D, const __nv_bfloat16* X, const float* V,
                              const SurPacked* model, float* w, float* f, double* f_soa, int* status,
                              int sms, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const long long ntiles = (n + TC_M - 1) / TC_M;
    // four CTAs per SM hold all 512 TMEM columns
    const long long grid = ntiles < 4ll * sms ? ntiles : 4ll * sms;
    if (X)
        k_sur_mlp_tc<true><<<(unsigned)grid, TC_M, 0, st>>>(n, nullptr, X, V, model, w, f, f_soa, status);
    else
        k_sur_mlp_tc<false><<<(unsigned)grid, TC_M, 0, st>>>(n, D, nullptr, V, model, w, f, f_soa, status);
    return cudaGetLastError();
}

}  // namespace atm3
