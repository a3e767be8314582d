// sur_train_tc.cu -- training of the surrogate MLP (32 -> 64 -> 64 -> 3, SiLU)
// on the fifth-generation tensor cores: forward and backward GEMMs as
// tcgen05.mma with bfloat16 operands in shared memory and FP32 accumulators
// in tensor memory (TMEM); FP32 master weights, FP32 gradients.
//
// One CTA of 128 threads per 128-sample tile (persistent over tiles); thread
// t owns sample t and TMEM lane t.  Per tile:
//   forward   Z1 = X W1, H1 = silu(Z1 + b1); Z2 = H1 W2, H2 = silu(Z2 + b2);
//             w = H2 W3 + b3 (the inference kernel's arithmetic: bfloat16
//             inputs, weights and hidden activations), F = sum_m w_m v_m
//   loss      L = norm sum |F - F_ref|^2, dL/dw_m = 2 norm (F - F_ref) . v_m
//   backward  dH2 = dY W3^T (CUDA cores, K = 3), dZ2 = dH2 silu'(Z2);
//             dH1 = dZ2 W2^T (tensor cores), dZ1 = dH1 silu'(Z1);
//             dW3 = H2^T dY, dW2 = H1^T dZ2, dW1 = X^T dZ1 (tensor cores,
//             contracting over the 128 samples), and the bias gradients
//             from the same GEMMs: the transposed left operands carry a row
//             of ones, whose output row is the column sum of the right one.
// silu'(z) (FP32) is kept in TMEM between the forward and the backward pass
// (tcgen05.st / tcgen05.ld).  The transposed operands (K = samples) are
// written element by element by the sample's thread.  Left operands of the
// weight gradients have M = 128 rows: rows beyond the weight rows and the
// ones row are zero.
//
// TMEM columns (256 per CTA, one CTA per SM by its shared memory):
//   [0, 64)    Z1 -> silu'(Z2) -> dH1
//   [64, 128)  Z2 -> dW2 (row 64: db2)
//   [128, 144) w
//   [144, 160) dW3 (row 64: db3)
//   [160, 224) silu'(Z1) -> dW1 (row 32: db1)
// Every wait on the MMA barrier is bounded; a wait that gives up stops the
// CTA (after freeing its TMEM) and sets ST_TIMEOUT.
#include <cuda_bf16.h>
#include <stdint.h>

#include "surrogate.cuh"
#include "tc_common.cuh"

namespace atm3 {

namespace {
using namespace tc;

constexpr int TR_M = 128;             // samples per tile = TMEM lanes
constexpr uint32_t TR_COLS = 256;     // TMEM columns per CTA
constexpr uint32_t SBO_K32 = 4 * 128, SBO_K64 = 8 * 128, SBO_K128 = 16 * 128;

struct TrSmem {
    alignas(128) unsigned char w1t[64 * 32 * 2];    // B, layer 1: N 64 x K 32 (W1^T)
    alignas(128) unsigned char w2t[64 * 64 * 2];    // B, layer 2: N 64 x K 64 (W2^T)
    alignas(128) unsigned char w3t[16 * 64 * 2];    // B, layer 3: N 16 x K 64 (W3^T)
    alignas(128) unsigned char w2[64 * 64 * 2];     // B of dH1 = dZ2 W2^T: N 64 (k) x K 64 (j)
    alignas(128) unsigned char x[TR_M * 32 * 2];    // A, layer 1: M 128 x K 32
    alignas(128) unsigned char h[TR_M * 64 * 2];    // A: H1 (layer 2), H2 (layer 3), dZ2 (dH1)
    alignas(128) unsigned char xt[128 * TR_M * 2];  // A of dW1: rows q < 32 X^T, row 32 ones
    alignas(128) unsigned char h1t[128 * TR_M * 2]; // A of dW2: rows k < 64 H1^T, row 64 ones
    alignas(128) unsigned char h2t[128 * TR_M * 2]; // A of dW3: rows k < 64 H2^T, row 64 ones
    alignas(128) unsigned char dyt[16 * TR_M * 2];  // B of dW3: N 16 (dL/dw_m) x K samples
    alignas(128) unsigned char dz2t[64 * TR_M * 2]; // B of dW2: N 64 x K samples
    alignas(128) unsigned char dz1t[64 * TR_M * 2]; // B of dW1: N 64 x K samples
    float w3[SUR_NH * SUR_NO];                      // FP32 master W3
    float b1[64], b2[64], b3[SUR_NO];
    double lsum[TR_M / 32];
    alignas(8) unsigned long long mbar;
    uint32_t tmem_base;
};

static_assert(sizeof(TrSmem) <= 227 * 1024, "one CTA's shared memory");

// element (row, k) of a K-major operand with kchunks 8-element chunks per row
__device__ __forceinline__ void put_bf(unsigned char* base, int row, int k, int kchunks, float v)
{
    *reinterpret_cast<__nv_bfloat16*>(base + cm_off(row, k >> 3, kchunks) + 2 * (k & 7)) =
        __float2bfloat16_rn(v);
}

// sigmoid and silu'(z) = s (1 + z (1 - s)); silu itself as the inference kernel forms it
__device__ __forceinline__ float sigm(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }

}  // namespace

namespace {

__global__ void __launch_bounds__(TR_M) k_sur_grad_tc(const SurGradArgs A)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    TrSmem& S = *reinterpret_cast<TrSmem*>(smraw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const SurPacked* model = A.packed;

    // ---- once per CTA: weights, constant rows of the padded operands, barrier, TMEM
    for (int e = tid; e < 64 * 4; e += TR_M) {
        const int r = e >> 2, j = e & 3;
        put_chunk(S.w1t, r, j, 4, *reinterpret_cast<const uint4*>(model->w1t + r * SUR_XS + 8 * j));
    }
    for (int e = tid; e < 64 * 8; e += TR_M) {
        const int r = e >> 3, j = e & 7;
        put_chunk(S.w2t, r, j, 8, *reinterpret_cast<const uint4*>(model->w2t + r * SUR_HS + 8 * j));
    }
    for (int e = tid; e < 16 * 8; e += TR_M) {
        const int r = e >> 3, j = e & 7;
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        put_chunk(S.w3t, r, j, 8, r < SUR_NO ? *reinterpret_cast<const uint4*>(model->w3t + r * SUR_HS + 8 * j) : z);
    }
    // W2 itself (row k holds W2[k][j], j contiguous) for dH1 = dZ2 W2^T
    for (int e = tid; e < SUR_NH * SUR_NH; e += TR_M)
        put_bf(S.w2, e >> 6, e & 63, 8, A.P[SUR_OFF_W2 + e]);
    for (int e = tid; e < SUR_NH * SUR_NO; e += TR_M) S.w3[e] = A.P[SUR_OFF_W3 + e];
    if (tid < 64) {
        S.b1[tid] = model->b1[tid];
        S.b2[tid] = model->b2[tid];
    }
    if (tid < SUR_NO) S.b3[tid] = model->b3[tid];
    {
        // zero rows of the padded left operands
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        for (int e = tid; e < (int)(sizeof(S.xt) / 16); e += TR_M) {
            reinterpret_cast<uint4*>(S.xt)[e] = z;
            reinterpret_cast<uint4*>(S.h1t)[e] = z;
            reinterpret_cast<uint4*>(S.h2t)[e] = z;
        }
        for (int e = tid; e < (int)(sizeof(S.dyt) / 16); e += TR_M) reinterpret_cast<uint4*>(S.dyt)[e] = z;
    }
    __syncthreads();
    // the rows of ones: their output rows are the bias gradients
    put_bf(S.xt, SUR_ND, tid, 16, 1.0f);
    put_bf(S.h1t, SUR_NH, tid, 16, 1.0f);
    put_bf(S.h2t, SUR_NH, tid, 16, 1.0f);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&S.tmem_base)),
                     "r"(TR_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;
    const uint32_t lane = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's lane quarter
    const uint32_t id64 = idesc_bf16(TR_M, 64), id16 = idesc_bf16(TR_M, 16);

    uint32_t phase = 0u;
    bool ok = true;
    // every thread waits on the MMA barrier's phase; all agree on the outcome
    auto wait_mma = [&]() {
        bool done = false;
        for (long it = 0; it < TC_WAIT_TRIES && !done; it++) done = mbar_try_wait(&S.mbar, phase);
        phase ^= 1u;
        ok = __syncthreads_and(done) != 0;
        tc_fence_after();
    };
    // operands written by the threads become visible to the tensor cores
    auto publish = [&]() {
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
    };
    // D (+)= A B over K / 16 instructions of K = 16
    auto mma = [&](uint32_t d, const unsigned char* a, const unsigned char* b, uint32_t sbo, int k,
                   uint32_t idesc) {
        for (int kk = 0; kk < k / 16; kk++)
            umma_bf16(d, sdesc(a + kk * 2 * TC_LBO, sbo), sdesc(b + kk * 2 * TC_LBO, sbo), idesc, kk > 0);
    };

    const long long ntiles = (A.batch + TR_M - 1) / TR_M;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long row = tile * TR_M + tid;
        const bool active = row < A.batch;
        const long long smp = active ? (A.idx ? A.idx[row] : row) : 0;

        // ---- inputs: normalised descriptors (X and X^T), vectors, target
        {
            float xv[SUR_ND];
#pragma unroll
            for (int q = 0; q < SUR_ND; q++)
                xv[q] = active ? (A.D[smp * SUR_ND + q] - A.mean[q]) / A.scale[q] : 0.0f;
#pragma unroll
            for (int j = 0; j < 4; j++)
                put_chunk(S.x, tid, j, 4,
                          make_uint4(pack_bf2(xv[8 * j], xv[8 * j + 1]), pack_bf2(xv[8 * j + 2], xv[8 * j + 3]),
                                     pack_bf2(xv[8 * j + 4], xv[8 * j + 5]), pack_bf2(xv[8 * j + 6], xv[8 * j + 7])));
#pragma unroll
            for (int q = 0; q < SUR_ND; q++) put_bf(S.xt, q, tid, 16, xv[q]);
        }
        float tg[3];
#pragma unroll
        for (int c = 0; c < 3; c++) tg[c] = active ? A.T[smp * 3 + c] : 0.0f;
        const float* vrow = A.V + smp * SUR_NV;  // the sample's 16 vectors (read when active)
        publish();

        // ---- layer 1: TMEM [0, 64) = X W1
        if (tid == 0) {
            tc_fence_after();
            mma(tmem, S.x, S.w1t, SBO_K32, SUR_ND, id64);
            umma_commit(&S.mbar);
        }
        wait_mma();
        if (!ok) break;
        // H1 = silu(Z1 + b1) into the layer-2 operand and H1^T; silu'(Z1) to TMEM [160, 224)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            float z[16], d[16];
            tmem_ld16(lane + 16 * q, z);
            uint32_t p[8];
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const int k = 16 * q + i;
                const float zb = z[i] + S.b1[k], s = sigm(zb);
                d[i] = s * (1.0f + zb * (1.0f - s));
                z[i] = silu(zb);
                put_bf(S.h1t, k, tid, 16, z[i]);
            }
#pragma unroll
            for (int i = 0; i < 8; i++) p[i] = pack_bf2(z[2 * i], z[2 * i + 1]);
            put_chunk(S.h, tid, 2 * q, 8, make_uint4(p[0], p[1], p[2], p[3]));
            put_chunk(S.h, tid, 2 * q + 1, 8, make_uint4(p[4], p[5], p[6], p[7]));
            tmem_st16(lane + 160 + 16 * q, d);
        }
        publish();

        // ---- layer 2: TMEM [64, 128) = H1 W2
        if (tid == 0) {
            tc_fence_after();
            mma(tmem + 64, S.h, S.w2t, SBO_K64, SUR_NH, id64);
            umma_commit(&S.mbar);
        }
        wait_mma();
        if (!ok) break;
        // H2 (over H1: layer 2 has read it), H2^T; silu'(Z2) to TMEM [0, 64)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            float z[16], d[16];
            tmem_ld16(lane + 64 + 16 * q, z);
            uint32_t p[8];
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const int k = 16 * q + i;
                const float zb = z[i] + S.b2[k], s = sigm(zb);
                d[i] = s * (1.0f + zb * (1.0f - s));
                z[i] = silu(zb);
                put_bf(S.h2t, k, tid, 16, z[i]);
            }
#pragma unroll
            for (int i = 0; i < 8; i++) p[i] = pack_bf2(z[2 * i], z[2 * i + 1]);
            put_chunk(S.h, tid, 2 * q, 8, make_uint4(p[0], p[1], p[2], p[3]));
            put_chunk(S.h, tid, 2 * q + 1, 8, make_uint4(p[4], p[5], p[6], p[7]));
            tmem_st16(lane + 16 * q, d);
        }
        publish();

        // ---- layer 3: TMEM [128, 144) = H2 W3
        if (tid == 0) {
            tc_fence_after();
            mma(tmem + 128, S.h, S.w3t, SBO_K64, SUR_NH, id16);
            umma_commit(&S.mbar);
        }
        wait_mma();
        if (!ok) break;
        double loss = 0.0;
        float dy[SUR_NO];
        {
            float o[16];
            tmem_ld16(lane + 128, o);
            float r[3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                float fc = 0.0f;
                if (active)
#pragma unroll
                    for (int m = 0; m < SUR_NO; m++) fc = fmaf(o[m] + S.b3[m], vrow[3 * m + c], fc);
                r[c] = fc - tg[c];
                loss += (double)r[c] * (double)r[c];
            }
            loss *= (double)A.norm;
            const float two_norm = 2.0f * A.norm;
#pragma unroll
            for (int m = 0; m < SUR_NO; m++) {
                dy[m] = active ? two_norm * (r[0] * vrow[3 * m] + r[1] * vrow[3 * m + 1] +
                                             r[2] * vrow[3 * m + 2])
                               : 0.0f;
                put_bf(S.dyt, m, tid, 16, dy[m]);
            }
        }
        // dZ2 = (dY W3^T) silu'(Z2) over H2 (layer 3 has read it) and into dZ2^T
#pragma unroll
        for (int q = 0; q < 4; q++) {
            float s2[16], dz[16];
            tmem_ld16(lane + 16 * q, s2);
            uint32_t p[8];
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const int k = 16 * q + i;
                float dh = 0.0f;
#pragma unroll
                for (int m = 0; m < SUR_NO; m++) dh = fmaf(dy[m], S.w3[SUR_NO * k + m], dh);
                dz[i] = dh * s2[i];
                put_bf(S.dz2t, k, tid, 16, dz[i]);
            }
#pragma unroll
            for (int i = 0; i < 8; i++) p[i] = pack_bf2(dz[2 * i], dz[2 * i + 1]);
            put_chunk(S.h, tid, 2 * q, 8, make_uint4(p[0], p[1], p[2], p[3]));
            put_chunk(S.h, tid, 2 * q + 1, 8, make_uint4(p[4], p[5], p[6], p[7]));
        }
        publish();

        // ---- dW3 (TMEM [144, 160)), dH1 (TMEM [0, 64)), dW2 (TMEM [64, 128))
        if (tid == 0) {
            tc_fence_after();
            mma(tmem + 144, S.h2t, S.dyt, SBO_K128, TR_M, id16);
            mma(tmem, S.h, S.w2, SBO_K64, SUR_NH, id64);
            mma(tmem + 64, S.h1t, S.dz2t, SBO_K128, TR_M, id64);
            umma_commit(&S.mbar);
        }
        wait_mma();
        if (!ok) break;
        // dZ1 = dH1 silu'(Z1) into dZ1^T
#pragma unroll
        for (int q = 0; q < 4; q++) {
            float dh[16], s1[16];
            tmem_ld16(lane + 16 * q, dh);
            tmem_ld16(lane + 160 + 16 * q, s1);
#pragma unroll
            for (int i = 0; i < 16; i++) put_bf(S.dz1t, 16 * q + i, tid, 16, dh[i] * s1[i]);
        }
        // gradient rows of layers 3 and 2 (TMEM lane = output row)
        float* G = A.part + tile * SUR_NP;
        {
            float o[16];
            tmem_ld16(lane + 144, o);
            if (tid < SUR_NH)
                for (int m = 0; m < SUR_NO; m++) G[SUR_OFF_W3 + tid * SUR_NO + m] = o[m];
            else if (tid == SUR_NH)
                for (int m = 0; m < SUR_NO; m++) G[SUR_OFF_B3 + m] = o[m];
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            float o[16];
            tmem_ld16(lane + 64 + 16 * q, o);
            if (tid < SUR_NH)
                for (int i = 0; i < 16; i++) G[SUR_OFF_W2 + tid * SUR_NH + 16 * q + i] = o[i];
            else if (tid == SUR_NH)
                for (int i = 0; i < 16; i++) G[SUR_OFF_B2 + 16 * q + i] = o[i];
        }
        publish();

        // ---- dW1 (TMEM [160, 224): silu'(Z1) has been read)
        if (tid == 0) {
            tc_fence_after();
            mma(tmem + 160, S.xt, S.dz1t, SBO_K128, TR_M, id64);
            umma_commit(&S.mbar);
        }
        wait_mma();
        if (!ok) break;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            float o[16];
            tmem_ld16(lane + 160 + 16 * q, o);
            if (tid < SUR_ND)
                for (int i = 0; i < 16; i++) G[SUR_OFF_W1 + tid * SUR_NH + 16 * q + i] = o[i];
            else if (tid == SUR_ND)
                for (int i = 0; i < 16; i++) G[SUR_OFF_B1 + 16 * q + i] = o[i];
        }
        // the tile's loss, in thread order
        for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
        if ((tid & 31) == 0) S.lsum[warp] = loss;
        tc_fence_before();
        __syncthreads();  // TMEM reads and operand reads done before the next tile
        tc_fence_after();
        if (tid == 0) A.part_loss[tile] = ((S.lsum[0] + S.lsum[1]) + S.lsum[2]) + S.lsum[3];
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TR_COLS)
                     : "memory");
    if (!ok && tid == 0) atomicOr(A.status, ST_TIMEOUT);
}

}  // namespace

int sur_grad_tc_tiles(long long batch) { return (int)((batch + TR_M - 1) / TR_M); }

cudaError_t launch_sur_grad_tc(const SurGradArgs& a, int sms, cudaStream_t st)
{
    const long long ntiles = (a.batch + TR_M - 1) / TR_M;
    if (ntiles <= 0) return cudaSuccess;
    const size_t smem = sizeof(TrSmem);
    cudaError_t e = cudaFuncSetAttribute(k_sur_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const long long grid = ntiles < (long long)sms ? ntiles : (long long)sms;
    k_sur_grad_tc<<<(unsigned)grid, TR_M, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace atm3
