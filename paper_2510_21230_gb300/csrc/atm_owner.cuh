// atm_owner.cuh -- owner-computes traversals: 3c01 (section 4) and the wide
// traversal 3cw (not in the paper: 5^3 cells, partners within R_w = 2 min w,
// third side below R_w too, which under the product rule finds the triplets
// the paper's traversals miss).
//
// One CTA per base cell.  The 27- (125-) cell neighbourhood is staged in
// shared memory; warps take the base cell's molecules i in turn.  For each i
// the warp builds i's partner list (pair rule: partners within r_c; product
// rule: every other staged molecule, 3cw: those within R_w) holding the
// displacement d(i -> q) and its square, then tests every pair {j, k} of the
// list and queues interacting pairs.  A full queue (32 pairs) is evaluated by the whole warp; only F_i is
// needed, so each lane keeps its share of F_i in registers (compensated in
// FP32) and the warp reduces it once per i: no atomics, deterministic.
// Energy and virial get u/3 and W/3 per visit (each triangle is found by up
// to three owners).
#pragma once
#include "atm_common.cuh"

namespace atm3 {

template <int TRAV, int TRUNC, typename R>
__device__ __forceinline__ void atm_owner_unit(const AtmArgs<R>& A, const long long u)
{
    constexpr int S = Trav<TRAV>::S;
    constexpr bool WIDE = TRAV == 3;
    constexpr bool F64 = sizeof(R) == 8;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_beg[S + 1];
    __shared__ int s_cell0[S];
    __shared__ signed char s_off[S][3];
    __shared__ int s_next;
    __shared__ unsigned long long s_cand;
    __shared__ double s_red[2][8];
    __shared__ unsigned long long s_redn[8];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int mcap = A.mcap;
    // the replica this unit belongs to and the unit's index inside it
    const Rep& rp = A.b.rep[A.b.rep_of_cell[u]];
    const long long lu = u - rp.cell0;
    const int pcap = A.pcap;
    const OwnerSmem plan = owner_smem_plan<R>(mcap, nwarps, pcap);
    R* px = reinterpret_cast<R*>(smem + plan.off_pos);
    R* py = px + mcap;
    R* pz = py + mcap;
    float* fx32 = F64 ? reinterpret_cast<float*>(smem + plan.off_pos32) : reinterpret_cast<float*>(px);
    float* fy32 = fx32 + mcap;
    float* fz32 = fy32 + mcap;
    unsigned char* sslot = smem + plan.off_slot;
    unsigned short* pq = reinterpret_cast<unsigned short*>(smem + plan.off_pq) + warp * pcap;
    R* pdx = reinterpret_cast<R*>(smem + plan.off_pd) + (size_t)warp * 4 * pcap;
    R* pdy = pdx + pcap;
    R* pdz = pdy + pcap;
    R* pa = pdz + pcap;
    float* pa32 = F64 ? reinterpret_cast<float*>(smem + plan.off_pa32) + warp * pcap : nullptr;
    unsigned* queue = reinterpret_cast<unsigned*>(smem + plan.off_queue) + warp * 64;

    if (!unit_owned(rp, lu)) {
        // another domain's base cell: its molecules get no owner force here
        if (tid == 0) {
            A.unit_ew[2 * u] = 0.0;
            A.unit_ew[2 * u + 1] = 0.0;
            A.unit_cnt[2 * u] = 0ull;
            A.unit_cnt[2 * u + 1] = 0ull;
        }
        const long long n = A.n;
        for (int g = A.cell_start[u] + tid; g < A.cell_start[u + 1]; g += blockDim.x) {
            A.fs[g] = 0.0;
            A.fs[n + g] = 0.0;
            A.fs[2 * n + g] = 0.0;
        }
        return;
    }
    if (warp == 0) unit_slots<TRAV, S>(rp.g, A.cell_start + rp.cell0, lu, s_beg, s_cell0, s_off);
    if (tid == 0) {
        s_next = 0;
        s_cand = 0ull;
    }
    __syncthreads();
    const int M = s_beg[S];
    const int Mfirst = s_beg[1];
    if (M > mcap) {
        if (tid == 0) {
            atomicOr(A.status, ST_CAPACITY);
            A.unit_ew[2 * u] = 0.0;
            A.unit_ew[2 * u + 1] = 0.0;
            A.unit_cnt[2 * u] = 0ull;
            A.unit_cnt[2 * u + 1] = 0ull;
        }
        return;
    }
    const long long n = A.n;
    for (int t = tid; t < M; t += blockDim.x) {
        // slot of staged molecule t: the last s with s_beg[s] <= t (a slot may be empty)
        int s = 0;
        if (S <= 32) {
            while (s_beg[s + 1] <= t) s++;
        } else {
            int hi = S - 1;
            while (s < hi) {
                const int mid = (s + hi + 1) >> 1;
                if (s_beg[mid] <= t) s = mid; else hi = mid - 1;
            }
        }
        int g = s_cell0[s] + (t - s_beg[s]);
        px[t] = A.xl[g];
        py[t] = A.xl[n + g];
        pz[t] = A.xl[2 * n + g];
        if (F64) {
            fx32[t] = A.xl32[g];
            fy32[t] = A.xl32[n + g];
            fz32[t] = A.xl32[2 * n + g];
        }
        sslot[t] = (unsigned char)s;
    }
    __syncthreads();

    const R w0 = (R)rp.g.w[0], w1 = (R)rp.g.w[1], w2 = (R)rp.g.w[2];
    const float wf0 = rp.wf[0], wf1 = rp.wf[1], wf2 = rp.wf[2];
    const R rc2 = F64 ? (R)rp.rc2 : (R)rp.rc2f;
    const R rc6 = F64 ? (R)rp.rc6 : (R)rp.rc6f;
    const R nu = F64 ? (R)rp.nu : (R)rp.nuf;
    const unsigned lt_mask = (1u << lane) - 1u;

    auto offs = [&](int p, int q, int& mx, int& my, int& mz) {
        int sp = sslot[p], sq = sslot[q];
        mx = s_off[sq][0] - s_off[sp][0];
        my = s_off[sq][1] - s_off[sp][1];
        mz = s_off[sq][2] - s_off[sp][2];
    };
    // squared distance decision p -> q under the pair rule (FP64 via the FP32 prefilter)
    auto close_pair = [&](int p, int q) -> bool {
        int mx, my, mz;
        offs(p, q, mx, my, mz);
        R dx, dy, dz;
        if (!F64) {
            R d2 = canon_disp<R>(px[p], py[p], pz[p], px[q], py[q], pz[q], mx, my, mz, w0, w1, w2,
                                 dx, dy, dz);
            return d2 < rc2;
        }
        float ex, ey, ez;
        float f2 = canon_disp<float>(fx32[p], fy32[p], fz32[p], fx32[q], fy32[q], fz32[q], mx, my,
                                     mz, wf0, wf1, wf2, ex, ey, ez);
        if (f2 < rp.p_lo) return true;
        if (f2 > rp.p_hi) return false;
        R d2 = canon_disp<R>(px[p], py[p], pz[p], px[q], py[q], pz[q], mx, my, mz, w0, w1, w2, dx,
                             dy, dz);
        return d2 < rc2;
    };

    // wide traversal: within R_w (FP32 decisions in FP32, FP64 ones in FP64)
    const R rw2 = F64 ? (R)rp.rw2 : (R)rp.rw2f;
    auto within_rw = [&](int p, int q) -> bool {
        int mx, my, mz;
        offs(p, q, mx, my, mz);
        R dx, dy, dz;
        return canon_disp<R>(px[p], py[p], pz[p], px[q], py[q], pz[q], mx, my, mz, w0, w1, w2, dx,
                             dy, dz) < rw2;
    };

    Sum<R> esum, wsum;
    unsigned int nint = 0;

    for (int it = 0;; it++) {
        // deterministic mode: warp w takes the molecules w, w + nwarps, ...
        // (so every lane's energy and virial sums repeat); else the next free one
        int i = it * nwarps + warp;
        if (!A.det) {
            if (lane == 0) i = atomicAdd(&s_next, 1);
            i = __shfl_sync(FULL, i, 0);
        }
        if (i >= Mfirst) break;

        // partner list of i: every other staged molecule (product) or those within r_c (pair)
        int np = 0;
        for (int q0 = 0; q0 < M; q0 += 32) {
            int q = q0 + lane;
            bool keep = false;
            if (q < M && q != i)
                keep = (TRUNC == 0) ? close_pair(i, q) : (WIDE ? within_rw(i, q) : true);
            unsigned m = __ballot_sync(FULL, keep);
            const int pos = np + __popc(m & lt_mask);
            if (keep && pos >= pcap) {
                atomicOr(A.status, ST_CAPACITY);  // more partners than the list holds
                keep = false;
            }
            if (keep) {
                int mx, my, mz;
                offs(i, q, mx, my, mz);
                R dx, dy, dz;
                R d2 = canon_disp<R>(px[i], py[i], pz[i], px[q], py[q], pz[q], mx, my, mz, w0, w1,
                                     w2, dx, dy, dz);
                pq[pos] = (unsigned short)q;
                pdx[pos] = dx;
                pdy[pos] = dy;
                pdz[pos] = dz;
                pa[pos] = d2;
                if (F64) {
                    float ex, ey, ez;
                    pa32[pos] = canon_disp<float>(fx32[i], fy32[i], fz32[i], fx32[q], fy32[q],
                                                  fz32[q], mx, my, mz, wf0, wf1, wf2, ex, ey, ez);
                }
            }
            np += __popc(m);
        }
        if (np > pcap) np = pcap;
        if (WIDE && lane == 0) atomicAdd(&s_cand, (unsigned long long)np * (unsigned long long)(np - 1) / 2ull);
        __syncwarp();

        Sum<R> fxs, fys, fzs;
        int qn = 0;
        auto evaluate = [&](unsigned e) {
            int jj = (int)(e & 0xffffu), kk = (int)(e >> 16);
            R dijx = pdx[jj], dijy = pdy[jj], dijz = pdz[jj], a = pa[jj];
            R dikx = pdx[kk], diky = pdy[kk], dikz = pdz[kk], b = pa[kk];
            R djkx = dikx - dijx, djky = diky - dijy, djkz = dikz - dijz;
            R c = djkx * djkx + djky * djky + djkz * djkz;
            R uu, ua, ub, uc;
            atm_terms<R>(a, b, c, nu, uu, ua, ub, uc);
            R gij = R(2) * ua, gik = R(2) * ub, gjk = R(2) * uc;
            esum.add(uu);
            wsum.add(-(gij * a + gik * b + gjk * c));
            fxs.add(gij * dijx + gik * dikx);
            fys.add(gij * dijy + gik * diky);
            fzs.add(gij * dijz + gik * dikz);
        };

        // pairs (jj < kk) of the partner list, kk-major (row kk holds jj = 0 ..
        // kk - 1), 32 per round: every lane walks from the warp's cursor
        // (kc, jc) to its own pair.  FP32 decides the third side j-k from the
        // partner vectors, d(j -> k) = d(i -> k) - d(i -> j): within 2.4e-4
        // (relative) of the canonical square for |d| above the guard
        // sqrt(dmin), so outside a band of 2^-10 around each threshold it
        // decides as the canonical form does; in the band, or below the
        // guard, the canonical displacement decides.
        const float bl = 1.0f - 0x1p-10f, bh = 1.0f + 0x1p-10f;
        int kc = 1, jc = 0;
        while (kc < np) {
            int kk = kc, jj = jc + lane;
            while (jj >= kk) {
                jj -= kk;
                kk++;
            }
            bool keep = false;
            if (kk < np) {
                int j = pq[jj], k = pq[kk];
                if (!F64) {
                    const float ex = (float)pdx[kk] - (float)pdx[jj];
                    const float ey = (float)pdy[kk] - (float)pdy[jj];
                    const float ez = (float)pdz[kk] - (float)pdz[jj];
                    const float cq = ex * ex + ey * ey + ez * ez;
                    const float a = (float)pa[jj], b = (float)pa[kk];
                    int state;  // 0 out, 1 in, 2 undecided
                    if (cq < rp.dmin) {
                        state = 2;
                    } else if (TRUNC == 0) {
                        state = cq < (float)rc2 * bl ? 1 : (cq > (float)rc2 * bh ? 0 : 2);
                    } else {
                        const float pr = (a * b) * cq;
                        state = pr < (float)rc6 * bl ? 1 : (pr > (float)rc6 * bh ? 0 : 2);
                        if (WIDE && state != 0)
                            state = cq > (float)rw2 * bh ? 0 : (cq < (float)rw2 * bl ? state : 2);
                    }
                    if (state == 2) {
                        if (TRUNC == 0) {
                            keep = close_pair(j, k);
                        } else {
                            int mx, my, mz;
                            offs(j, k, mx, my, mz);
                            R dx, dy, dz;
                            R c = canon_disp<R>(px[j], py[j], pz[j], px[k], py[k], pz[k], mx, my,
                                                mz, w0, w1, w2, dx, dy, dz);
                            keep = (!WIDE || c < rw2) && sorted_product<R>(pa[jj], pa[kk], c) < rc6;
                        }
                    } else {
                        keep = state == 1;
                    }
                } else if (TRUNC == 0) {
                    keep = close_pair(j, k);
                } else if (WIDE) {
                    // third side below R_w, then the sorted product, in the working precision
                    int mx, my, mz;
                    offs(j, k, mx, my, mz);
                    R dx, dy, dz;
                    R c = canon_disp<R>(px[j], py[j], pz[j], px[k], py[k], pz[k], mx, my, mz, w0,
                                        w1, w2, dx, dy, dz);
                    keep = c < rw2 && sorted_product<R>(pa[jj], pa[kk], c) < rc6;
                } else {
                    int mx, my, mz;
                    offs(j, k, mx, my, mz);
                    float ex, ey, ez;
                    float a32 = pa32[jj], b32 = pa32[kk];
                    float c32 = canon_disp<float>(fx32[j], fy32[j], fz32[j], fx32[k], fy32[k],
                                                  fz32[k], mx, my, mz, wf0, wf1, wf2, ex, ey, ez);
                    float pr = sorted_product<float>(a32, b32, c32);
                    float lo = fminf(a32, fminf(b32, c32));
                    if (lo >= rp.dmin && pr < rp.q_lo) {
                        keep = true;
                    } else if (lo >= rp.dmin && pr > rp.q_hi) {
                        keep = false;
                    } else {
                        R dx, dy, dz;
                        R c = canon_disp<R>(px[j], py[j], pz[j], px[k], py[k], pz[k], mx, my, mz,
                                            w0, w1, w2, dx, dy, dz);
                        keep = sorted_product<R>(pa[jj], pa[kk], c) < rc6;
                    }
                }
            }
            unsigned m = __ballot_sync(FULL, keep);
            if (keep) queue[qn + __popc(m & lt_mask)] = (unsigned)jj | ((unsigned)kk << 16);
            qn += __popc(m);
            nint += keep ? 1u : 0u;
            __syncwarp();
            if (qn >= 32) {
                evaluate(queue[lane]);
                __syncwarp();
                if (lane < qn - 32) queue[lane] = queue[32 + lane];
                qn -= 32;
                __syncwarp();
            }
            jc += 32;  // the next cursor (uniform)
            while (jc >= kc) {
                jc -= kc;
                kc++;
            }
        }
        if (lane < qn) evaluate(queue[lane]);
        // F_i: lane shares combined in FP64
        double f0 = fxs.get(), f1 = fys.get(), f2 = fzs.get();
        for (int o = 16; o > 0; o >>= 1) {
            f0 += __shfl_down_sync(FULL, f0, o);
            f1 += __shfl_down_sync(FULL, f1, o);
            f2 += __shfl_down_sync(FULL, f2, o);
        }
        if (lane == 0) {
            int g = s_cell0[0] + i;  // base slot comes first: staged index = offset in the base cell
            A.fs[g] = f0;
            A.fs[n + g] = f1;
            A.fs[2 * n + g] = f2;
        }
        __syncwarp();
    }

    unsigned long long cand = 0;
    if (WIDE) __syncthreads();  // every warp's partner-pair count is in
    if (tid == 0) {
        if constexpr (WIDE) cand = s_cand;
        else cand = unit_candidates<TRAV, S>(s_beg);
    }
    unit_reduce_store<8>(esum.get(), wsum.get(), (unsigned long long)nint, 1.0 / 3.0, cand,
                         A.unit_ew, A.unit_cnt, u, s_red, s_redn);
}

// One CTA per base cell, or (A.work set) a persistent grid pulling units from
// a global counter.
template <int TRAV, int TRUNC, typename R>
__global__ void __launch_bounds__(128) atm_owner_kernel(const AtmArgs<R> A)
{
    if (A.work == nullptr) {
        atm_owner_unit<TRAV, TRUNC, R>(A, blockIdx.x);
        return;
    }
    __shared__ int s_u;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_u = atomicAdd(A.work, 1);
        __syncthreads();
        const int u = s_u;
        if (u >= A.b.ncell) break;
        atm_owner_unit<TRAV, TRUNC, R>(A, u);
    }
}

}  // namespace atm3
