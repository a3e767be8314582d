// sur_kernels.cu -- kernels of the learned ATM force surrogate (model in
// surrogate.cuh): descriptors, bfloat16 tensor-core MLP + force assembly,
// data-set collection, FP32 training gradient, Adam, statistics.
#include <cuda_bf16.h>
#include <stdint.h>

#include "surrogate.cuh"

namespace atm3 {

namespace {

constexpr int SUR_BLOCK = 128;  // molecules per CTA of the descriptor kernel
constexpr float SUR_R0 = 0.8f;
constexpr float SUR_PI = 3.14159265358979f;

// ------------------------------------------------------------ descriptors

// descriptor accumulators of one molecule (registers: every index is static)
struct SurAcc {
    float G[16];    // radial channels
    float p[4][3];  // vector moments
    float T[3][6];  // traceless quadrupole moments xx yy zz xy xz yz
};

// Every channel has eta d^2 = 1/2, so with u = (r - mu_0) / d the channel-j
// Gaussian is exp(-(u - j)^2 / 2) = 2^(-((u - j) s)^2), s = sqrt(log2(e) / 2):
// one subtraction of an immediate, one square and one base-2 exponential.
constexpr float SUR_SQH = 0.8493218002880191f;  // sqrt(log2(e) / 2)

struct SurConst {
    float rc2, sg, sv, pi_rc;  // sg = s / d_g, sv = s / d_v
};

__device__ __forceinline__ SurConst sur_consts(const Rep& rp)
{
    SurConst k;
    const float rc = rp.rcf;
    k.rc2 = rp.rc2f;
    k.sg = SUR_SQH / ((rc - SUR_R0) / 15.0f);
    k.sv = SUR_SQH / ((rc - SUR_R0) / 4.0f);
    k.pi_rc = SUR_PI / rc;
    return k;
}

// 2^x (hardware approximation; x <= 0 here, results below the FP32 normal
// range flush to zero)
__device__ __forceinline__ float sur_exp2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void sur_zero(SurAcc& a)
{
#pragma unroll
    for (int k = 0; k < 16; k++) a.G[k] = 0.0f;
#pragma unroll
    for (int m = 0; m < 4; m++) a.p[m][0] = a.p[m][1] = a.p[m][2] = 0.0f;
#pragma unroll
    for (int m = 0; m < 3; m++)
#pragma unroll
        for (int c = 0; c < 6; c++) a.T[m][c] = 0.0f;
}

// one neighbour at displacement (ex, ey, ez), r2 = |e|^2 < r_c^2
__device__ __forceinline__ void sur_add(SurAcc& a, const SurConst& k, float ex, float ey, float ez,
                                        float r2)
{
    const float ir = rsqrtf(r2);
    const float r = r2 * ir;
    const float ux = ex * ir, uy = ey * ir, uz = ez * ir;
    const float fc = 0.5f * (__cosf(k.pi_rc * r) + 1.0f);
    const float rr = r - SUR_R0;
    const float vg = rr * k.sg;  // (r - mu_0) s / d_g
#pragma unroll
    for (int j = 0; j < 16; j++) {
        const float tt = vg - (float)j * SUR_SQH;
        a.G[j] += sur_exp2(-(tt * tt)) * fc;
    }
    const float vv = rr * k.sv - 0.5f * SUR_SQH;  // (r - nu_0) s / d_v
    const float third = 1.0f / 3.0f;
    const float qxx = ux * ux - third, qyy = uy * uy - third, qzz = uz * uz - third;
    const float qxy = ux * uy, qxz = ux * uz, qyz = uy * uz;
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const float tt = vv - (float)m * SUR_SQH;
        const float ph = sur_exp2(-(tt * tt)) * fc;
        a.p[m][0] += ph * ux;
        a.p[m][1] += ph * uy;
        a.p[m][2] += ph * uz;
        if (m < 3) {
            a.T[m][0] += ph * qxx;
            a.T[m][1] += ph * qyy;
            a.T[m][2] += ph * qzz;
            a.T[m][3] += ph * qxy;
            a.T[m][4] += ph * qxz;
            a.T[m][5] += ph * qyz;
        }
    }
}

constexpr int SUR_MW = 32;  // candidate-mask words per molecule: 1024 candidates of its 27 cells

// ---------------------------------------------------------------- kernels

__global__ void __launch_bounds__(256) k_sur_xyz4(long long n, const float* __restrict__ xl,
                                                  float4* __restrict__ xl4)
{
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s < n) xl4[s] = make_float4(xl[s], xl[n + s], xl[2 * n + s], 0.0f);
}

// One thread per sorted molecule.  Descriptors in two passes: (A) every
// candidate of the molecule's 27 cells is tested against the cutoff and
// recorded as one bit (cheap, so lanes in different cells diverge little);
// (B) the thread walks its set bits and accumulates the descriptor terms, so
// the expensive part keeps every lane busy.  More than 1024 candidates: one
// direct pass.  With LJ the same neighbours give the FP32 LJ pair force,
// energy, virial and counts of the molecule (the decisions and arithmetic of
// the FP32 LJ kernel, so no separate LJ pass is needed).  Mode 0 writes the
// normalised bfloat16 input row and the
// vectors for the MLP kernel; mode 1 appends the raw descriptors, vectors and
// the current ATM force to the data set.  The masks are word-major (word w of
// thread t at w * SUR_BLOCK + t), free of bank conflicts.
template <bool LJ>
__global__ void __launch_bounds__(SUR_BLOCK, 5) k_sur_desc(const SurForceArgs A)
{
    __shared__ unsigned mask[SUR_MW * SUR_BLOCK];
    // per thread and neighbour cell t: end of t's candidates in the bit order
    // and q - k for t's candidates ([t][thread], free of bank conflicts)
    __shared__ int s_kend[27 * SUR_BLOCK];
    __shared__ int s_qoff[27 * SUR_BLOCK];
    const int tid = threadIdx.x;
    const long long n = A.n;
    const long long s = (long long)blockIdx.x * SUR_BLOCK + tid;
    if (s >= n) return;
    const int cg = A.cell_sorted[s];
    const Rep& rp = A.b.rep[A.b.rep_of_cell[cg]];
    int cx, cy, cz;
    cell_coords(rp.g, cg - rp.cell0, cx, cy, cz);
    const int* st = A.cell_start + rp.cell0;
    const SurConst kc = sur_consts(rp);
    const float4* __restrict__ x4 = A.xl4;
    const float4 xs = x4[s];
    SurAcc acc;
    sur_zero(acc);
    // (A) candidate k of the concatenated 27 cells -> bit k (the molecule itself
    // passes the test; its bit is cleared below)
    // displacement and squared distance rounded as written (no contraction):
    // the cutoff decisions are those of the FP32 LJ kernel
    auto dist2 = [&](const float4& xq, float sx, float sy, float sz, float& ex, float& ey,
                     float& ez) -> float {
        ex = __fadd_rn(__fsub_rn(xq.x, xs.x), sx);
        ey = __fadd_rn(__fsub_rn(xq.y, xs.y), sy);
        ez = __fadd_rn(__fsub_rn(xq.z, xs.z), sz);
        return __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
    };
    // LJ of one neighbour (the FP32 LJ kernel's expressions)
    float ljx = 0.f, ljy = 0.f, ljz = 0.f, lje = 0.f, ljw = 0.f;
    unsigned lj_cand = 0u, lj_pairs = 0u;
    // fwd: the neighbour is in the forward half shell (a later molecule of the
    // own cell, or a forward cell), so the pair is counted once, here
    auto lj_add = [&](float ex, float ey, float ez, float a, bool fwd) {
        const float ia = __frcp_rn(a);  // correctly rounded: the same value as 1 / a
        const float s2 = rp.sig2f * ia;
        const float s3 = s2 * s2 * s2;
        const float s6 = s3 * s3;
        const float fw = (rp.eps48f * s6 - rp.eps24f * s3) * ia;
        ljx -= fw * ex;
        ljy -= fw * ey;
        ljz -= fw * ez;
        lje += rp.eps4f * (s6 - s3) - rp.ushiftf;
        ljw += fw * a;
        lj_pairs += fwd ? 1u : 0u;
    };
    int K = 0, kself = 0;
    unsigned word = 0u;
    for (int t = 0; t < 27; t++) {
        int dx, dy, dz;
        offset27(t, dx, dy, dz);
        const long long nc = cell_at(rp.g, cx, cy, cz, dx, dy, dz);
        const int q0 = st[nc], q1 = st[nc + 1];
        if (t == 13) kself = K + (int)(s - q0);
        if (LJ) {
            if (t > 13) lj_cand += (unsigned)(q1 - q0);
            if (t == 13) lj_cand += (unsigned)(q1 - 1 - s);
        }
        s_kend[t * SUR_BLOCK + tid] = K + (q1 - q0);
        s_qoff[t * SUR_BLOCK + tid] = q0 - K;
        const float sx = (float)dx * rp.wf[0], sy = (float)dy * rp.wf[1], sz = (float)dz * rp.wf[2];
        for (int q = q0; q < q1; q++) {
            float ex, ey, ez;
            const float r2 = dist2(x4[q], sx, sy, sz, ex, ey, ez);
            word |= (r2 < kc.rc2 ? 1u : 0u) << (K & 31);
            K++;
            if ((K & 31) == 0) {
                if (K <= 32 * SUR_MW) mask[((K >> 5) - 1) * SUR_BLOCK + tid] = word;
                word = 0u;
            }
        }
    }
    if ((K & 31) != 0 && K < 32 * SUR_MW) mask[(K >> 5) * SUR_BLOCK + tid] = word;
    if (K <= 32 * SUR_MW) {
        mask[(kself >> 5) * SUR_BLOCK + tid] &= ~(1u << (kself & 31));
        // (B) one iteration per set bit (not per mask word), so every lane
        // runs as many iterations as it has neighbours
        const int nw = (K + 31) >> 5;
        int t = 0, w = -1;
        unsigned bits = 0u;
        for (;;) {
            while (bits == 0u && ++w < nw) bits = mask[w * SUR_BLOCK + tid];
            if (bits == 0u) break;
            const int k = (w << 5) + __ffs(bits) - 1;
            bits &= bits - 1u;
            while (k >= s_kend[t * SUR_BLOCK + tid]) t++;
            int dx, dy, dz;
            offset27(t, dx, dy, dz);
            float ex, ey, ez;
            const int q = k + s_qoff[t * SUR_BLOCK + tid];
            const float r2 = dist2(x4[q], (float)dx * rp.wf[0], (float)dy * rp.wf[1],
                                   (float)dz * rp.wf[2], ex, ey, ez);
            sur_add(acc, kc, ex, ey, ez, r2);
            if (LJ) lj_add(ex, ey, ez, r2, t > 13 || (t == 13 && q > s));
        }
    } else {
        // crowded neighbourhood: test and accumulate in one pass
        for (int t = 0; t < 27; t++) {
            int dx, dy, dz;
            offset27(t, dx, dy, dz);
            const long long nc = cell_at(rp.g, cx, cy, cz, dx, dy, dz);
            const int q0 = st[nc], q1 = st[nc + 1];
            const float sx = (float)dx * rp.wf[0], sy = (float)dy * rp.wf[1], sz = (float)dz * rp.wf[2];
            for (int q = q0; q < q1; q++) {
                if (q == s) continue;
                float ex, ey, ez;
                const float r2 = dist2(x4[q], sx, sy, sz, ex, ey, ez);
                if (r2 < kc.rc2) {
                    sur_add(acc, kc, ex, ey, ez, r2);
                    if (LJ) lj_add(ex, ey, ez, r2, t > 13 || (t == 13 && q > s));
                }
            }
        }
    }
    if (LJ) {
        A.f_lj[s] = (double)ljx;
        A.f_lj[n + s] = (double)ljy;
        A.f_lj[2 * n + s] = (double)ljz;
        A.mol_ew[2 * s] = 0.5 * (double)lje;
        A.mol_ew[2 * s + 1] = 0.5 * (double)ljw;
        A.mol_cnt[2 * s] = lj_cand;
        A.mol_cnt[2 * s + 1] = lj_pairs;
    }
    // the invariants, streamed out eight at a time: raw FP32 (mode 1) or
    // normalised bfloat16 in 16-byte stores (mode 0)
    const bool collect = A.mode == 1;
    const long long row = A.row0 + s;
    const float* mean = A.model ? A.model->mean : nullptr;
    const float* scale = A.model ? A.model->scale : nullptr;
    float buf[8];
    auto put = [&](int k, float dk) {
        buf[k & 7] = dk;
        if ((k & 7) != 7) return;
        const int k0 = k - 7;
        if (collect) {
            float4* d = reinterpret_cast<float4*>(A.d_out + row * SUR_ND + k0);
            d[0] = make_float4(buf[0], buf[1], buf[2], buf[3]);
            d[1] = make_float4(buf[4], buf[5], buf[6], buf[7]);
        } else {
            uint32_t h[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                __nv_bfloat162 b2 = __floats2bfloat162_rn((buf[2 * j] - mean[k0 + 2 * j]) / scale[k0 + 2 * j],
                                                          (buf[2 * j + 1] - mean[k0 + 2 * j + 1]) /
                                                              scale[k0 + 2 * j + 1]);
                h[j] = *reinterpret_cast<uint32_t*>(&b2);
            }
            unsigned char* tile = reinterpret_cast<unsigned char*>(A.xb + (s / SUR_TILE_M) * (SUR_TILE_M * SUR_ND));
            *reinterpret_cast<uint4*>(tile + sur_tile_off((int)(s % SUR_TILE_M), k0 >> 3, SUR_ND / 8)) =
                make_uint4(h[0], h[1], h[2], h[3]);
        }
    };
#pragma unroll
    for (int k = 0; k < 16; k++) put(k, acc.G[k]);
    int e = 16;
#pragma unroll
    for (int m = 0; m < 4; m++)
#pragma unroll
        for (int b = m; b < 4; b++)
            put(e++, acc.p[m][0] * acc.p[b][0] + acc.p[m][1] * acc.p[b][1] + acc.p[m][2] * acc.p[b][2]);
#pragma unroll
    for (int m = 0; m < 3; m++)
#pragma unroll
        for (int b = m; b < 3; b++)
            put(e++, acc.T[m][0] * acc.T[b][0] + acc.T[m][1] * acc.T[b][1] + acc.T[m][2] * acc.T[b][2] +
                         2.0f * (acc.T[m][3] * acc.T[b][3] + acc.T[m][4] * acc.T[b][4] +
                                 acc.T[m][5] * acc.T[b][5]));
    // the 16 equivariant vectors: p_0..p_3, then T_a p_b (a < 3, b < 4) with
    // T stored as (xx, yy, zz, xy, xz, yz); twelve 16-byte stores of a row
    float vv[SUR_NV];
#pragma unroll
    for (int m = 0; m < 4; m++) {
        vv[3 * m] = acc.p[m][0];
        vv[3 * m + 1] = acc.p[m][1];
        vv[3 * m + 2] = acc.p[m][2];
    }
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const float* T = acc.T[a];
            const float* p = acc.p[b];
            const int m = 4 + 4 * a + b;
            vv[3 * m] = T[0] * p[0] + T[3] * p[1] + T[4] * p[2];
            vv[3 * m + 1] = T[3] * p[0] + T[1] * p[1] + T[5] * p[2];
            vv[3 * m + 2] = T[4] * p[0] + T[5] * p[1] + T[2] * p[2];
        }
    float4* v4 = reinterpret_cast<float4*>(collect ? A.v_out + row * SUR_NV : A.vb + s * SUR_NV);
#pragma unroll
    for (int q = 0; q < SUR_NV / 4; q++)
        v4[q] = make_float4(vv[4 * q], vv[4 * q + 1], vv[4 * q + 2], vv[4 * q + 3]);
    if (collect) {
        float* t = A.t_out + row * 3;
        t[0] = (float)A.f_atm[s];
        t[1] = (float)A.f_atm[n + s];
        t[2] = (float)A.f_atm[2 * n + s];
    }
}

// ------------------------------------------------------------- training

constexpr int GH = 65;                 // row stride of the 64-wide FP32 tiles
constexpr int GX = 33;                 // row stride of the input tile
constexpr int SUR_NP_PAD = (SUR_NP + 3) & ~3;

struct GradSmem {
    static constexpr int P = 0;
    static constexpr int W2T = P + SUR_NP_PAD;          // W2 transposed [j][k]
    static constexpr int X = W2T + SUR_NH * SUR_NH;
    static constexpr int H1 = X + SUR_TILE * GX;
    static constexpr int S1 = H1 + SUR_TILE * GH;       // silu'(z1), then dL/dz1
    static constexpr int H2 = S1 + SUR_TILE * GH;
    static constexpr int S2 = H2 + SUR_TILE * GH;       // silu'(z2), then dL/dz2
    static constexpr int V = S2 + SUR_TILE * GH;
    static constexpr int T = V + SUR_TILE * SUR_NV;
    static constexpr int W = T + SUR_TILE * 3;          // outputs w, then dL/dw [i][SUR_NO]
    static constexpr int END = W + SUR_TILE * SUR_NO;
};
constexpr size_t SUR_GRAD_SMEM = GradSmem::END * sizeof(float) + SUR_TILE * sizeof(double);

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + expf(-z)); }

__global__ void __launch_bounds__(SUR_GRAD_THREADS) k_sur_grad(const SurGradArgs A)
{
    extern __shared__ __align__(16) float sm[];
    float* P = sm + GradSmem::P;
    float* W2T = sm + GradSmem::W2T;
    float* X = sm + GradSmem::X;
    float* H1 = sm + GradSmem::H1;
    float* S1 = sm + GradSmem::S1;
    float* H2 = sm + GradSmem::H2;
    float* S2 = sm + GradSmem::S2;
    float* Vs = sm + GradSmem::V;
    float* Ts = sm + GradSmem::T;
    float* Wt = sm + GradSmem::W;
    double* Ls = reinterpret_cast<double*>(sm + GradSmem::END);
    const int tid = threadIdx.x;
    const long long base = (long long)blockIdx.x * SUR_TILE;

    for (int k = tid; k < SUR_NP; k += SUR_GRAD_THREADS) P[k] = A.P[k];
    for (int k = tid; k < SUR_NH * SUR_NH; k += SUR_GRAD_THREADS) {
        const int kk = k / SUR_NH, j = k % SUR_NH;
        W2T[j * SUR_NH + kk] = A.P[SUR_OFF_W2 + k];
    }
    for (int e = tid; e < SUR_TILE * SUR_ND; e += SUR_GRAD_THREADS) {
        const int i = e / SUR_ND, q = e % SUR_ND;
        const long long row = base + i;
        float x = 0.0f;
        if (row < A.batch) {
            const long long smp = A.idx ? A.idx[row] : row;
            x = (A.D[smp * SUR_ND + q] - A.mean[q]) / A.scale[q];
        }
        X[i * GX + q] = x;
    }
    for (int e = tid; e < SUR_TILE * SUR_NV; e += SUR_GRAD_THREADS) {
        const int i = e / SUR_NV, q = e % SUR_NV;
        const long long row = base + i;
        Vs[e] = row < A.batch ? A.V[(A.idx ? A.idx[row] : row) * SUR_NV + q] : 0.0f;
    }
    for (int e = tid; e < SUR_TILE * 3; e += SUR_GRAD_THREADS) {
        const int i = e / 3, q = e % 3;
        const long long row = base + i;
        Ts[e] = row < A.batch ? A.T[(A.idx ? A.idx[row] : row) * 3 + q] : 0.0f;
    }
    __syncthreads();

    // thread tile of the 64 x 64 products: rows rg + 0..3, columns cg + 16 c
    const int rg = (tid >> 4) * 4, cg = tid & 15;

    // layer 1: z1 = X W1 + b1
    {
        float z[4][4];
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) z[r][c] = P[SUR_OFF_B1 + cg + 16 * c];
        for (int q = 0; q < SUR_ND; q++) {
            float xa[4], wb[4];
#pragma unroll
            for (int r = 0; r < 4; r++) xa[r] = X[(rg + r) * GX + q];
#pragma unroll
            for (int c = 0; c < 4; c++) wb[c] = P[SUR_OFF_W1 + q * SUR_NH + cg + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) z[r][c] = fmaf(xa[r], wb[c], z[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const float zz = z[r][c], sg = sigm(zz);
                H1[(rg + r) * GH + cg + 16 * c] = zz * sg;
                S1[(rg + r) * GH + cg + 16 * c] = sg * (1.0f + zz * (1.0f - sg));
            }
    }
    __syncthreads();
    // layer 2: z2 = H1 W2 + b2
    {
        float z[4][4];
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) z[r][c] = P[SUR_OFF_B2 + cg + 16 * c];
        for (int k = 0; k < SUR_NH; k++) {
            float ha[4], wb[4];
#pragma unroll
            for (int r = 0; r < 4; r++) ha[r] = H1[(rg + r) * GH + k];
#pragma unroll
            for (int c = 0; c < 4; c++) wb[c] = P[SUR_OFF_W2 + k * SUR_NH + cg + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) z[r][c] = fmaf(ha[r], wb[c], z[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const float zz = z[r][c], sg = sigm(zz);
                H2[(rg + r) * GH + cg + 16 * c] = zz * sg;
                S2[(rg + r) * GH + cg + 16 * c] = sg * (1.0f + zz * (1.0f - sg));
            }
    }
    __syncthreads();
    // outputs w = H2 W3 + b3
    for (int e = tid; e < SUR_TILE * SUR_NO; e += SUR_GRAD_THREADS) {
        const int i = e / SUR_NO, m = e % SUR_NO;
        float acc = P[SUR_OFF_B3 + m];
        for (int k = 0; k < SUR_NH; k++) acc = fmaf(H2[i * GH + k], P[SUR_OFF_W3 + k * SUR_NO + m], acc);
        Wt[i * SUR_NO + m] = acc;
    }
    __syncthreads();
    // residuals, loss and dL/dw (padding rows have V = T = 0: no contribution)
    if (tid < SUR_TILE) {
        const int i = tid;
        const float* v = Vs + i * SUR_NV;
        const float* wi = Wt + i * SUR_NO;
        float r[3];
        double l = 0.0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            float fc = 0.0f;
            for (int m = 0; m < SUR_NO; m++) fc = fmaf(wi[m], v[3 * m + c], fc);
            r[c] = fc - Ts[i * 3 + c];
            l += (double)r[c] * (double)r[c];
        }
        Ls[i] = l * (double)A.norm;
        const float two_norm = 2.0f * A.norm;
        for (int m = 0; m < SUR_NO; m++)
            Wt[i * SUR_NO + m] = two_norm * (r[0] * v[3 * m] + r[1] * v[3 * m + 1] + r[2] * v[3 * m + 2]);
    }
    __syncthreads();
    float* G = A.part + (long long)blockIdx.x * SUR_NP;
    if (tid == 0) {
        double l = 0.0;
        for (int i = 0; i < SUR_TILE; i++) l += Ls[i];
        A.part_loss[blockIdx.x] = l;
    }
    // output layer gradient; dL/dz2 = silu'(z2) * (W3 dL/dw)
    for (int e = tid; e < SUR_NH * SUR_NO + SUR_NO; e += SUR_GRAD_THREADS) {
        if (e < SUR_NH * SUR_NO) {
            const int k = e / SUR_NO, m = e % SUR_NO;
            float acc = 0.0f;
            for (int i = 0; i < SUR_TILE; i++) acc = fmaf(H2[i * GH + k], Wt[i * SUR_NO + m], acc);
            G[SUR_OFF_W3 + k * SUR_NO + m] = acc;
        } else {
            const int m = e - SUR_NH * SUR_NO;
            float acc = 0.0f;
            for (int i = 0; i < SUR_TILE; i++) acc += Wt[i * SUR_NO + m];
            G[SUR_OFF_B3 + m] = acc;
        }
    }
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int i = rg + r, k = cg + 16 * c;
            float dh = 0.0f;
            for (int m = 0; m < SUR_NO; m++) dh = fmaf(P[SUR_OFF_W3 + k * SUR_NO + m], Wt[i * SUR_NO + m], dh);
            S2[i * GH + k] *= dh;
        }
    __syncthreads();
    // second layer gradient; dL/dz1 = silu'(z1) * (W2 dL/dz2)
    {
        float g[4][4];
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) g[r][c] = 0.0f;
        for (int i = 0; i < SUR_TILE; i++) {
            float ha[4], db[4];
#pragma unroll
            for (int r = 0; r < 4; r++) ha[r] = H1[i * GH + rg + r];
#pragma unroll
            for (int c = 0; c < 4; c++) db[c] = S2[i * GH + cg + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) g[r][c] = fmaf(ha[r], db[c], g[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) G[SUR_OFF_W2 + (rg + r) * SUR_NH + cg + 16 * c] = g[r][c];
    }
    if (tid < SUR_NH) {
        float acc = 0.0f;
        for (int i = 0; i < SUR_TILE; i++) acc += S2[i * GH + tid];
        G[SUR_OFF_B2 + tid] = acc;
    }
    {
        float d[4][4];
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) d[r][c] = 0.0f;
        for (int j = 0; j < SUR_NH; j++) {
            float da[4], wb[4];
#pragma unroll
            for (int r = 0; r < 4; r++) da[r] = S2[(rg + r) * GH + j];
#pragma unroll
            for (int c = 0; c < 4; c++) wb[c] = W2T[j * SUR_NH + cg + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) d[r][c] = fmaf(da[r], wb[c], d[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) S1[(rg + r) * GH + cg + 16 * c] *= d[r][c];
    }
    __syncthreads();
    // first layer gradient: rows q = 2 (tid >> 4) + 0..1 of W1
    {
        const int qg = (tid >> 4) * 2;
        float g[2][4];
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) g[r][c] = 0.0f;
        for (int i = 0; i < SUR_TILE; i++) {
            float xa[2], db[4];
#pragma unroll
            for (int r = 0; r < 2; r++) xa[r] = X[i * GX + qg + r];
#pragma unroll
            for (int c = 0; c < 4; c++) db[c] = S1[i * GH + cg + 16 * c];
#pragma unroll
            for (int r = 0; r < 2; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) g[r][c] = fmaf(xa[r], db[c], g[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) G[SUR_OFF_W1 + (qg + r) * SUR_NH + cg + 16 * c] = g[r][c];
    }
    if (tid < SUR_NH) {
        float acc = 0.0f;
        for (int i = 0; i < SUR_TILE; i++) acc += S1[i * GH + tid];
        G[SUR_OFF_B1 + tid] = acc;
    }
}

// packed inference slot of master parameter k
__device__ __forceinline__ void pack_param(SurPacked* Pk, int k, float val)
{
    if (k < SUR_OFF_B1) {
        Pk->w1t[(k % SUR_NH) * SUR_XS + k / SUR_NH] = __float2bfloat16_rn(val);
    } else if (k < SUR_OFF_W2) {
        Pk->b1[k - SUR_OFF_B1] = val;
    } else if (k < SUR_OFF_B2) {
        const int e = k - SUR_OFF_W2;
        Pk->w2t[(e % SUR_NH) * SUR_HS + e / SUR_NH] = __float2bfloat16_rn(val);
    } else if (k < SUR_OFF_W3) {
        Pk->b2[k - SUR_OFF_B2] = val;
    } else if (k < SUR_OFF_B3) {
        const int e = k - SUR_OFF_W3;
        Pk->w3t[(e % SUR_NO) * SUR_HS + e / SUR_NO] = __float2bfloat16_rn(val);
    } else {
        Pk->b3[k - SUR_OFF_B3] = val;
    }
}

// gradient = sum of the CTA parts in CTA order; Adam (Kingma & Ba, Algorithm 1)
__global__ void __launch_bounds__(256) k_sur_adam(const SurAdamArgs A)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0 && A.loss_out) {
        double l = 0.0;
        for (int c = 0; c < A.nct; c++) l += A.part_loss[c];
        *A.loss_out = l;
    }
    if (k >= SUR_NP) return;
    float g = 0.0f;
    for (int c = 0; c < A.nct; c++) g += A.part[(long long)c * SUR_NP + k];
    if (A.grad_out) A.grad_out[k] = g;
    if (!A.update) return;
    const float m = A.beta1 * A.m[k] + (1.0f - A.beta1) * g;
    const float v = A.beta2 * A.v[k] + (1.0f - A.beta2) * g * g;
    A.m[k] = m;
    A.v[k] = v;
    const float p = A.P[k] - A.lr * (m / A.c1) / (sqrtf(v / A.c2) + A.eps);
    A.P[k] = p;
    pack_param(A.packed, k, p);
}

__global__ void k_sur_pack(const float* P, const float* mean, const float* scale, SurPacked* Pk)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < SUR_NP) pack_param(Pk, k, P[k]);
    if (k < SUR_ND) {
        Pk->mean[k] = mean[k];
        Pk->scale[k] = scale[k];
    }
}

// splitmix64 output function (Steele, Lea & Flood 2014) of a (seed, step, b) counter
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_sur_sample(long long* idx, long long batch, long long S, unsigned long long seed,
                             long long step)
{
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= batch) return;
    unsigned long long z = mix64(seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(step + 1));
    z = mix64(z + 0x9E3779B97F4A7C15ull * (unsigned long long)(b + 1));
    idx[b] = (long long)(z % (unsigned long long)S);
}

// column sums of a fixed chunk of rows per CTA (deterministic order)
__global__ void __launch_bounds__(256) k_sur_stats(const float* __restrict__ D,
                                                   const float* __restrict__ T, long long S,
                                                   const double* center, int square,
                                                   double* part)
{
    __shared__ double red[8][SUR_ND + 1];
    const int tid = threadIdx.x, col = tid & 31, grp = tid >> 5;
    const long long lo = S * blockIdx.x / SUR_STAT_PARTS, hi = S * (blockIdx.x + 1) / SUR_STAT_PARTS;
    const double c = center ? center[col] : 0.0;
    double acc = 0.0, acc_t = 0.0;
    for (long long i = lo + grp; i < hi; i += 8) {
        const double d = (double)D[i * SUR_ND + col] - c;
        acc += square ? d * d : d;
        if (col < 3) acc_t += (double)T[i * 3 + col] * (double)T[i * 3 + col];
    }
    red[grp][col] = acc;
    // |T|^2 per group: lanes 0..2 add their component in lane order
    const double t1 = __shfl_sync(0xffffffffu, acc_t, 1), t2 = __shfl_sync(0xffffffffu, acc_t, 2);
    if (col == 0) red[grp][SUR_ND] = (acc_t + t1) + t2;
    __syncthreads();
    if (tid <= SUR_ND) {
        double s = 0.0;
        for (int g = 0; g < 8; g++) s += red[g][tid];
        part[blockIdx.x * (SUR_ND + 1) + tid] = s;
    }
}

__global__ void __launch_bounds__(256) k_sur_diff(long long n, const double* __restrict__ a,
                                                  const double* __restrict__ b, double* acc)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double d2 = 0.0, b2 = 0.0;
    if (i < n)
        for (int c = 0; c < 3; c++) {
            const double d = a[c * n + i] - b[c * n + i];
            d2 += d * d;
            b2 += b[c * n + i] * b[c * n + i];
        }
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_down_sync(0xffffffffu, d2, o);
        b2 += __shfl_down_sync(0xffffffffu, b2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, d2);
        atomicAdd(acc + 1, b2);
    }
}

unsigned blocks_of(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t launch_sur_forces(const SurForceArgs& a, cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    k_sur_xyz4<<<blocks_of(a.n, 256), 256, 0, st>>>(a.n, a.xl32, a.xl4);
    if (a.f_lj)
        k_sur_desc<true><<<blocks_of(a.n, SUR_BLOCK), SUR_BLOCK, 0, st>>>(a);
    else
        k_sur_desc<false><<<blocks_of(a.n, SUR_BLOCK), SUR_BLOCK, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.mode != 0) return e;
    return launch_sur_mlp_tc(a.n, nullptr, a.xb, a.vb, a.model, nullptr, nullptr, a.f_atm, a.status,
                             a.sms, st);
}

cudaError_t launch_sur_mlp_rows(long long n, const float* D, const float* V, const SurPacked* model,
                                float* w, float* f, int* status, int sms, cudaStream_t st)
{
    return launch_sur_mlp_tc(n, D, nullptr, V, model, w, f, nullptr, status, sms, st);
}

cudaError_t launch_sur_grad(const SurGradArgs& a, int nct, cudaStream_t st)
{
    if (nct <= 0) return cudaSuccess;
    // per device; cheap enough to repeat on every launch
    cudaError_t e = cudaFuncSetAttribute(k_sur_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SUR_GRAD_SMEM);
    if (e != cudaSuccess) return e;
    k_sur_grad<<<nct, SUR_GRAD_THREADS, SUR_GRAD_SMEM, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sur_adam(const SurAdamArgs& a, cudaStream_t st)
{
    k_sur_adam<<<blocks_of(SUR_NP, 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sur_pack(const float* P, const float* mean, const float* scale, SurPacked* packed,
                            cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(packed, 0, sizeof(SurPacked), st);
    if (e != cudaSuccess) return e;
    k_sur_pack<<<blocks_of(SUR_NP, 256), 256, 0, st>>>(P, mean, scale, packed);
    return cudaGetLastError();
}

cudaError_t launch_sur_sample(long long* idx, long long batch, long long S, unsigned long long seed,
                              long long step, cudaStream_t st)
{
    if (batch <= 0 || S <= 0) return cudaSuccess;
    k_sur_sample<<<blocks_of(batch, 256), 256, 0, st>>>(idx, batch, S, seed, step);
    return cudaGetLastError();
}

cudaError_t launch_sur_stats(const float* D, const float* T, long long S, const double* center,
                             int square, double* part, cudaStream_t st)
{
    k_sur_stats<<<SUR_STAT_PARTS, 256, 0, st>>>(D, T, S, center, square, part);
    return cudaGetLastError();
}

cudaError_t launch_sur_diff(long long n, const double* a, const double* b, double* acc,
                            cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_sur_diff<<<blocks_of(n, 256), 256, 0, st>>>(n, a, b, acc);
    return cudaGetLastError();
}

}  // namespace atm3
