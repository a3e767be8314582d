// surrogate.cuh -- learned per-molecule model of the ATM three-body force:
// device types and host launchers of sur_kernels.cu.
//
// Model (the library's own; the paper evaluates the triplet sum exactly):
//   neighbours j of i with r = |r_j - r_i| < r_c, rhat = (r_j - r_i) / r,
//   cutoff f_c(r) = (cos(pi r / r_c) + 1) / 2;
//   16 radial channels G_k = sum_j exp(-eta_g (r - mu_k)^2) f_c,
//      mu_k = 0.8 + k d_g, d_g = (r_c - 0.8) / 15, eta_g = 1 / (2 d_g^2);
//   4 vector channels phi_a = exp(-eta_v (r - nu_a)^2) f_c,
//      nu_a = 0.8 + (a + 1/2) d_v, d_v = (r_c - 0.8) / 4, eta_v = 1 / (2 d_v^2),
//      p_a = sum_j phi_a rhat, T_a = sum_j phi_a (rhat rhat^T - I/3) (a < 3);
//   descriptors D = [G_0..15, p_a.p_b (ab = 00 01 02 03 11 12 13 22 23 33),
//                    tr(T_a T_b) (ab = 00 01 02 11 12 22)];
//   MLP xn = (D - mean) / scale -> silu(xn W1 + b1) -> silu(. W2 + b2) -> w = . W3 + b3;
//   F_i = sum_{m<3} w_m p_m.
// Inference runs in bfloat16 on the tcgen05 tensor cores with FP32
// accumulation in tensor memory (inputs, weights and the two hidden
// activations rounded to bfloat16); training runs in FP32 on FP32 master
// weights.
#pragma once
#include <cuda_bf16.h>

#include "atm3_internal.cuh"

namespace atm3 {

constexpr int SUR_ND = 32;   // descriptors
constexpr int SUR_NH = 64;   // hidden width
constexpr int SUR_NO = 16;   // outputs (weights of the 16 vectors)
constexpr int SUR_NV = 48;   // 16 3-vectors: p_0..p_3, then T_a p_b (a < 3, b < 4)
constexpr int SUR_OFF_W1 = 0;
constexpr int SUR_OFF_B1 = SUR_OFF_W1 + SUR_ND * SUR_NH;
constexpr int SUR_OFF_W2 = SUR_OFF_B1 + SUR_NH;
constexpr int SUR_OFF_B2 = SUR_OFF_W2 + SUR_NH * SUR_NH;
constexpr int SUR_OFF_W3 = SUR_OFF_B2 + SUR_NH;
constexpr int SUR_OFF_B3 = SUR_OFF_W3 + SUR_NH * SUR_NO;
constexpr int SUR_NP = SUR_OFF_B3 + SUR_NO;  // 7312

// row strides (bf16 elements) of the packed weight rows: 16-byte multiples,
// so the tensor-core kernel stages them in 16-byte chunks
constexpr int SUR_XS = 40;   // K = 32 rows
constexpr int SUR_HS = 72;   // K = 64 rows

// Inference weights in bfloat16, n-major with k contiguous (row n holds the
// weights into output n), padded rows; FP32 biases and the descriptor
// normalisation.
struct SurPacked {
    __nv_bfloat16 w1t[SUR_NH * SUR_XS];
    __nv_bfloat16 w2t[SUR_NH * SUR_HS];
    __nv_bfloat16 w3t[SUR_NO * SUR_HS];
    float b1[SUR_NH], b2[SUR_NH], b3[SUR_NO];
    float mean[SUR_ND], scale[SUR_ND];
};
static_assert(sizeof(SurPacked) % 16 == 0, "SurPacked is copied in 16-byte pieces");

// Tiles of 128 rows for the tensor-core MLP.  The normalised bfloat16 input
// rows are stored tile by tile in the tensor cores' canonical K-major layout
// without swizzle (8-row x 16-byte core matrices; core matrix (row group g,
// 8-element chunk j) at byte g * (K / 8) * 128 + j * 128, row r of it at
// + 16 r), so one bulk copy moves a tile into shared memory as is.
constexpr int SUR_TILE_M = 128;
__host__ __device__ constexpr unsigned sur_tile_off(int row, int chunk, int kchunks)
{
    return (unsigned)((row >> 3) * (kchunks * 128) + chunk * 128 + (row & 7) * 16);
}

struct SurForceArgs {
    Batch b;
    long long n;              // SoA stride = b.ntot
    const float* xl32;        // sorted cell-local FP32 coordinates, SoA [3n]
    const int* cell_start;    // [ncell + 1]
    const int* cell_sorted;   // [n]
    const SurPacked* model;
    double* f_atm;            // [3n] sorted order: surrogate force (mode 0)
    // scratch owned by the caller: packed coordinates [n] (both modes),
    // normalised bfloat16 descriptor tiles [ceil(n/128)][128 x 32] (tile
    // layout above) and vectors [ceil(n/128) * 128][9] (mode 0)
    float4* xl4;
    __nv_bfloat16* xb;
    float* vb;
    // LJ pair forces from the same neighbour pass (FP32, owner computes, the
    // arithmetic of the FP32 LJ kernel); nullptr: not computed
    double* f_lj;             // [3n] sorted order
    double* mol_ew;           // [2n] half pair energies and virials per molecule
    unsigned* mol_cnt;        // [2n] half-shell candidates, visits
    int* status;              // device status word (ST_TIMEOUT)
    int sms;                  // SMs of the device (persistent MLP grid)
    // mode 1 (collect): raw descriptors, vectors and the current f_atm as the
    // training target, rows [row0, row0 + n) of the data set (sorted order)
    float* d_out;             // [.][32]
    float* v_out;             // [.][9]
    float* t_out;             // [.][3]
    long long row0;
    int mode;
};

// training: FP32 forward + backward of one minibatch; CTA c handles the
// samples idx[64 c .. 64 c + 63] (< batch), writes its gradient part[c][SUR_NP]
// and loss part_loss[c] (sum of squared residuals * norm)
struct SurGradArgs {
    const float* D;           // [S][32] raw descriptors
    const float* V;           // [S][9]
    const float* T;           // [S][3] target forces
    const long long* idx;     // [batch] sample rows (nullptr: rows 0..batch-1)
    long long batch;
    const float* P;           // [SUR_NP] FP32 master parameters
    const float* mean;        // [32]
    const float* scale;       // [32]
    float norm;               // 1 / (3 batch sigma2)
    float* part;              // [nct][SUR_NP]
    double* part_loss;        // [nct]
    // tensor-core training: the bfloat16 inference copy of the weights (the
    // forward pass) and the device status word (ST_TIMEOUT)
    const SurPacked* packed;
    int* status;
};

constexpr int SUR_TILE = 64;      // samples per CTA of the training kernel
constexpr int SUR_GRAD_THREADS = 256;

struct SurAdamArgs {
    const float* part;        // [nct][SUR_NP]
    const double* part_loss;  // [nct]
    int nct;
    float* P;                 // master parameters (updated when update != 0)
    float* m;
    float* v;
    const float* mean;
    const float* scale;
    SurPacked* packed;        // inference copy (written when update != 0)
    float* grad_out;          // optional [SUR_NP] summed gradient
    double* loss_out;         // optional loss of this step
    int update;
    float lr, beta1, beta2, eps, c1, c2;  // c1 = 1 - beta1^t, c2 = 1 - beta2^t
};

// descriptors (and, mode 0, the MLP and the force): three launches
cudaError_t launch_sur_forces(const SurForceArgs& a, cudaStream_t st);
constexpr int SUR_LAUNCHES = 3;
// MLP on given descriptor rows (no neighbour search): w[n][3], f[n][3]
cudaError_t launch_sur_mlp_rows(long long n, const float* D, const float* V,
                                const SurPacked* model, float* w, float* f, int* status, int sms,
                                cudaStream_t st);
// the MLP on the tcgen05 tensor cores (sur_tc.cu): input raw FP32 rows D or
// normalised bfloat16 tiles X (tile layout, padded to whole tiles like V),
// vectors V; outputs any of w[n][3], f[n][3] and f_soa [3][n] (FP64); a wait
// that gives up sets ST_TIMEOUT in *status
cudaError_t launch_sur_mlp_tc(long long n, const float* D, const __nv_bfloat16* X, const float* V,
                              const SurPacked* model, float* w, float* f, double* f_soa, int* status,
                              int sms, cudaStream_t st);
cudaError_t launch_sur_grad(const SurGradArgs& a, int nct, cudaStream_t st);
// the same gradient on the tensor cores (bfloat16 operands, FP32 accumulators):
// one part per 128-sample tile, sur_grad_tc_tiles(batch) parts
cudaError_t launch_sur_grad_tc(const SurGradArgs& a, int sms, cudaStream_t st);
int sur_grad_tc_tiles(long long batch);
cudaError_t launch_sur_adam(const SurAdamArgs& a, cudaStream_t st);
// pack FP32 master parameters + normalisation into the inference layout
cudaError_t launch_sur_pack(const float* P, const float* mean, const float* scale,
                            SurPacked* packed, cudaStream_t st);
// minibatch rows: idx[b] = splitmix64(seed, step, b) mod S
cudaError_t launch_sur_sample(long long* idx, long long batch, long long S, unsigned long long seed,
                              long long step, cudaStream_t st);
// partial sums over 256 fixed chunks of the data set: part[c][0..31] = sum of
// (D - center) or (D - center)^2 (square != 0), part[c][32] = sum |T|^2
cudaError_t launch_sur_stats(const float* D, const float* T, long long S, const double* center,
                             int square, double* part, cudaStream_t st);
constexpr int SUR_STAT_PARTS = 256;
// sum of |a - b|^2 and |b|^2 over SoA [3n] FP64 arrays, added to acc[0..1]
cudaError_t launch_sur_diff(long long n, const double* a, const double* b, double* acc,
                            cudaStream_t st);

}  // namespace atm3
