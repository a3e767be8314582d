// atm_block.cuh -- Newton-3 traversals 3c18 and 3c08 (section 4).
//
// One CTA per unit: the base cell with its 13 forward neighbours (3c18) or
// the 2x2x2 block anchored at the base cell (3c08).  The unit's M molecules
// are staged in shared memory in slot order, so a triplet i < j < k of staged
// indices always lists its cells in the order the traversal's tasks do.
//
//  1. Pair decisions.  Pair rule: an upper-triangular bitmask adjacency
//     adj[p] = {q > p : |d(p,q)| < r_c} (one ballot per 32 pairs) and its
//     transpose; edges are numbered row by row.  Product rule: a dense table
//     of FP32 squared distances (or on-the-fly distances when it does not fit).
//  2. Triangles.  Pair rule: for every first molecule p and edge (p,q), the
//     third molecules are the set bits of adj[p] & adj[q] & (allowed slots),
//     i.e. the triplet's three pair tests are shared by every triplet that
//     contains the pair.  Product rule: every candidate p < q < r of the
//     unit's tasks is tested on the sorted product of its squared sides.
//     Interacting triplets go to a warp queue and are evaluated 32 at a time.
//  3. Edge scalars.  By Eq. forcepairs each triplet's forces are three pair
//     terms g_e d_e along its sides (g = 2 du/d(r^2)), so a triplet adds three
//     scalars to per-pair accumulators G_e instead of nine force components.
//  4. Gather.  Every molecule m sums F_m = sum_e G_e d(m -> other end) over
//     its pairs in one thread (compensated in FP32), and adds the unit's share
//     to the global FP64 force once.
#pragma once
#include "atm_common.cuh"

namespace atm3 {

__device__ __forceinline__ int tri_index(int x, int y) { return y * (y - 1) / 2 + x; }  // x < y

template <int TRAV, int TRUNC, typename R>
__global__ void __launch_bounds__(256) atm_block_kernel(const AtmArgs<R> A)
{
    constexpr int S = Trav<TRAV>::S;
    constexpr bool F64 = sizeof(R) == 8;
    constexpr bool PAIR = TRUNC == 0;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_beg[S + 1];
    __shared__ int s_cell0[S];
    __shared__ signed char s_off[S][3];
    __shared__ int s_next, s_edges;
    __shared__ double s_red[2][8];
    __shared__ unsigned long long s_redn[8];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const long long u = blockIdx.x;
    const int mcap = A.mcap;
    const BlockSmem plan = block_smem_plan<R>(TRUNC, mcap, nwarps, A.gcap, A.use_d);
    const int W = plan.W;
    R* px = reinterpret_cast<R*>(smem + plan.off_pos);
    R* py = px + mcap;
    R* pz = py + mcap;
    float* fx32 = F64 ? reinterpret_cast<float*>(smem + plan.off_pos32) : reinterpret_cast<float*>(px);
    float* fy32 = fx32 + mcap;
    float* fz32 = fy32 + mcap;
    int* sidx = reinterpret_cast<int*>(smem + plan.off_idx);
    unsigned char* sslot = smem + plan.off_slot;
    unsigned* adj = reinterpret_cast<unsigned*>(smem + plan.off_adj);
    unsigned* adjT = reinterpret_cast<unsigned*>(smem + plan.off_adjT);
    int* rowoff = reinterpret_cast<int*>(smem + plan.off_rowoff);
    unsigned* memb = reinterpret_cast<unsigned*>(smem + plan.off_memb);
    R* G = reinterpret_cast<R*>(smem + plan.off_G);
    float* D = reinterpret_cast<float*>(smem + plan.off_D);
    unsigned short* plq = reinterpret_cast<unsigned short*>(smem + plan.off_plq) + warp * mcap;
    unsigned long long* queue =
        reinterpret_cast<unsigned long long*>(smem + plan.off_queue) + warp * 64;

    if (warp == 0) unit_slots<TRAV, S>(A.g, A.cell_start, u, s_beg, s_cell0, s_off);
    if (tid == 0) s_next = 0;
    __syncthreads();
    const int M = s_beg[S];
    const int Mfirst = (TRAV == 2) ? M : s_beg[1];
    const int npair = M * (M - 1) / 2;
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
    const int Wm = (M + 31) >> 5;
    const long long n = A.n;

    // ---- stage the unit
    for (int t = tid; t < M; t += blockDim.x) {
        int s = 0;
        while (s_beg[s + 1] <= t) s++;
        int g = s_cell0[s] + (t - s_beg[s]);
        px[t] = A.xl[g];
        py[t] = A.xl[n + g];
        pz[t] = A.xl[2 * n + g];
        if (F64) {
            fx32[t] = A.xl32[g];
            fy32[t] = A.xl32[n + g];
            fz32[t] = A.xl32[2 * n + g];
        }
        sidx[t] = g;
        sslot[t] = (unsigned char)s;
    }
    const int gsize = PAIR ? A.gcap : npair;
    for (int t = tid; t < gsize; t += blockDim.x) G[t] = R(0);
    if (PAIR)
        for (int t = tid; t < M * W; t += blockDim.x) adjT[t] = 0u;
    __syncthreads();

    const R w0 = A.w[0], w1 = A.w[1], w2 = A.w[2];
    const float wf0 = A.wf[0], wf1 = A.wf[1], wf2 = A.wf[2];
    const R rc2 = A.rc2, rc6 = A.rc6, nu = A.nu;
    const unsigned lt_mask = (1u << lane) - 1u;

    auto offs = [&](int p, int q, int& mx, int& my, int& mz) {
        int sp = sslot[p], sq = sslot[q];
        mx = s_off[sq][0] - s_off[sp][0];
        my = s_off[sq][1] - s_off[sp][1];
        mz = s_off[sq][2] - s_off[sp][2];
    };
    auto disp = [&](int p, int q, R& dx, R& dy, R& dz) -> R {
        int mx, my, mz;
        offs(p, q, mx, my, mz);
        return canon_disp<R>(px[p], py[p], pz[p], px[q], py[q], pz[q], mx, my, mz, w0, w1, w2, dx,
                             dy, dz);
    };
    auto disp32 = [&](int p, int q) -> float {
        int mx, my, mz;
        offs(p, q, mx, my, mz);
        float dx, dy, dz;
        return canon_disp<float>(fx32[p], fy32[p], fz32[p], fx32[q], fy32[q], fz32[q], mx, my, mz,
                                 wf0, wf1, wf2, dx, dy, dz);
    };

    // ---- 1. pair decisions
    if (PAIR) {
        for (int p = warp; p < M; p += nwarps) {
            for (int w = 0; w < (p >> 5); w++)
                if (lane == 0) adj[p * W + w] = 0u;
            for (int w = p >> 5; w < Wm; w++) {
                int q = (w << 5) + lane;
                bool keep = false;
                if (q > p && q < M) {
                    if (!F64) {
                        R dx, dy, dz;
                        keep = disp(p, q, dx, dy, dz) < rc2;
                    } else {
                        float f2 = disp32(p, q);
                        if (f2 < A.p_lo) {
                            keep = true;
                        } else if (f2 <= A.p_hi) {
                            R dx, dy, dz;
                            keep = disp(p, q, dx, dy, dz) < rc2;
                        }
                    }
                }
                unsigned word = __ballot_sync(FULL, keep);
                if (lane == 0) adj[p * W + w] = word;
                if (keep) atomicOr(&adjT[q * W + (p >> 5)], 1u << (p & 31));
            }
        }
    } else if (A.use_d) {
        for (int t = tid; t < npair; t += blockDim.x) {
            int y = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)t)) * 0.5f);
            while (y * (y - 1) / 2 > t) y--;
            while ((y + 1) * y / 2 <= t) y++;
            int x = t - y * (y - 1) / 2;
            D[t] = disp32(x, y);
        }
    }
    __syncthreads();
    if (PAIR) {
        if (warp == 0) {
            int run = 0;
            for (int p0 = 0; p0 < M; p0 += 32) {
                int p = p0 + lane;
                int c = 0;
                if (p < M)
                    for (int w = 0; w < Wm; w++) c += __popc(adj[p * W + w]);
                int incl = c;
                for (int o = 1; o < 32; o <<= 1) {
                    int v = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += v;
                }
                if (p < M) rowoff[p] = run + incl - c;
                run += __shfl_sync(FULL, incl, 31);
            }
            if (lane == 0) {
                rowoff[M] = run;
                s_edges = run;
            }
        }
        if (TRAV == 2) {
            // molecules r allowed as third member given v = slot(p) & slot(q): (v & slot(r)) == 0
            for (int t = tid; t < 8 * Wm; t += blockDim.x) {
                int v = t / Wm, w = t - v * Wm;
                unsigned word = 0u;
                for (int b = 0; b < 32; b++) {
                    int r = (w << 5) + b;
                    if (r < M && (v & sslot[r]) == 0) word |= 1u << b;
                }
                memb[v * W + w] = word;
            }
        }
        __syncthreads();
        if (s_edges > A.gcap) {
            if (tid == 0) {
                atomicOr(A.status, ST_CAPACITY);
                A.unit_ew[2 * u] = 0.0;
                A.unit_ew[2 * u + 1] = 0.0;
                A.unit_cnt[2 * u] = 0ull;
                A.unit_cnt[2 * u + 1] = 0ull;
            }
            return;
        }
    }

    // rank of y among the set bits of row x (edges of x are numbered in bit order)
    auto rank = [&](int x, int y) -> int {
        int wy = y >> 5, c = 0;
        for (int w = 0; w < wy; w++) c += __popc(adj[x * W + w]);
        return c + __popc(adj[x * W + wy] & ((1u << (y & 31)) - 1u));
    };

    // ---- 2 + 3. triangles, evaluation, edge scalars
    Sum<R> esum, wsum;
    unsigned int nint = 0;
    int qn = 0;

    auto evaluate = [&](unsigned long long e) {
        int p = (int)(e & 0x7ff), q = (int)((e >> 11) & 0x7ff), r = (int)((e >> 22) & 0x7ff);
        int jj = (int)((e >> 33) & 0x7ff);
        R dpqx, dpqy, dpqz, dprx, dpry, dprz, dqrx, dqry, dqrz;
        R a = disp(p, q, dpqx, dpqy, dpqz);
        R b = disp(p, r, dprx, dpry, dprz);
        R c = disp(q, r, dqrx, dqry, dqrz);
        R uu, ua, ub, uc;
        atm_terms<R>(a, b, c, nu, uu, ua, ub, uc);
        R gpq = R(2) * ua, gpr = R(2) * ub, gqr = R(2) * uc;
        esum.add(uu);
        wsum.add(-(gpq * a + gpr * b + gqr * c));
        int epq, epr, eqr;
        if (PAIR) {
            epq = rowoff[p] + jj;
            epr = rowoff[p] + rank(p, r);
            eqr = rowoff[q] + rank(q, r);
        } else {
            epq = tri_index(p, q);
            epr = tri_index(p, r);
            eqr = tri_index(q, r);
        }
        atomicAdd(G + epq, gpq);
        atomicAdd(G + epr, gpr);
        atomicAdd(G + eqr, gqr);
    };
    auto push = [&](bool keep, unsigned long long entry) {
        unsigned m = __ballot_sync(FULL, keep);
        if (keep) queue[qn + __popc(m & lt_mask)] = entry;
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
    };
    auto pack = [](int p, int q, int r, int jj) -> unsigned long long {
        return (unsigned long long)p | ((unsigned long long)q << 11) |
               ((unsigned long long)r << 22) | ((unsigned long long)jj << 33);
    };

    for (;;) {
        int p = 0;
        if (lane == 0) p = atomicAdd(&s_next, 1);
        p = __shfl_sync(FULL, p, 0);
        if (p >= Mfirst) break;
        const int sp = sslot[p];
        if (TRAV == 2 && sp == 7) continue;  // no later slot completes an anchored set
        if (PAIR) {
            // edges (p, q), q > p, in bit order
            int np = 0;
            for (int w = p >> 5; w < Wm; w++) {
                unsigned word = adj[p * W + w];
                if ((word >> lane) & 1u) plq[np + __popc(word & lt_mask)] = (unsigned short)((w << 5) + lane);
                np += __popc(word);
            }
            __syncwarp();
            for (int c0 = 0; c0 < np; c0 += 32) {
                const int jj = c0 + lane;
                const bool act = jj < np;
                const int q = act ? plq[jj] : 0;
                const int v = act ? (sp & sslot[q]) : 0;
                int w = q >> 5;
                unsigned cur = 0u;
                if (act)
                    cur = adj[p * W + w] & adj[q * W + w] & (TRAV == 2 ? memb[v * W + w] : FULL);
                for (;;) {
                    if (act)
                        while (cur == 0u && w + 1 < Wm) {
                            w++;
                            cur = adj[p * W + w] & adj[q * W + w] &
                                  (TRAV == 2 ? memb[v * W + w] : FULL);
                        }
                    const bool has = act && cur != 0u;
                    if (!__any_sync(FULL, has)) break;
                    int r = 0;
                    if (has) {
                        r = (w << 5) + __ffs(cur) - 1;
                        cur &= cur - 1u;
                    }
                    push(has, pack(p, q, r, jj));
                }
            }
        } else {
            // every candidate p < q < r of the unit's tasks
            const int base = p + 1, L = M - base;
            const int T = L * (L - 1) / 2;
            for (int t0 = 0; t0 < T; t0 += 32) {
                int t = t0 + lane;
                bool keep = false;
                int q = 0, r = 0;
                if (t < T) {
                    int kk = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)t)) * 0.5f);
                    while (kk * (kk - 1) / 2 > t) kk--;
                    while ((kk + 1) * kk / 2 <= t) kk++;
                    int jj = t - kk * (kk - 1) / 2;
                    q = base + jj;
                    r = base + kk;
                    bool member = (TRAV != 2) || ((sp & sslot[q] & sslot[r]) == 0);
                    if (member) {
                        float a32, b32, c32;
                        if (A.use_d) {
                            a32 = D[tri_index(p, q)];
                            b32 = D[tri_index(p, r)];
                            c32 = D[tri_index(q, r)];
                        } else {
                            a32 = disp32(p, q);
                            b32 = disp32(p, r);
                            c32 = disp32(q, r);
                        }
                        float pr = sorted_product<float>(a32, b32, c32);
                        if (!F64) {
                            keep = pr < (float)rc6;
                        } else {
                            float lo = fminf(a32, fminf(b32, c32));
                            if (lo >= A.dmin && pr < A.q_lo) {
                                keep = true;
                            } else if (lo >= A.dmin && pr > A.q_hi) {
                                keep = false;
                            } else {
                                R dx, dy, dz;
                                R a = disp(p, q, dx, dy, dz);
                                R b = disp(p, r, dx, dy, dz);
                                R c = disp(q, r, dx, dy, dz);
                                keep = sorted_product<R>(a, b, c) < rc6;
                            }
                        }
                    }
                }
                push(keep, pack(p, q, r, 0));
            }
        }
        __syncwarp();
    }
    if (lane < qn) evaluate(queue[lane]);
    __syncthreads();

    // ---- 4. gather: F_m = sum over m's pairs of G_e d(m -> other end)
    for (int m = tid; m < M; m += blockDim.x) {
        Sum<R> fxs, fys, fzs;
        auto add_pair = [&](int y, R g) {
            if (g == R(0)) return;
            R dx, dy, dz;
            disp(m, y, dx, dy, dz);
            fxs.add(g * dx);
            fys.add(g * dy);
            fzs.add(g * dz);
        };
        if (PAIR) {
            int e = rowoff[m];
            for (int w = 0; w < Wm; w++) {
                unsigned up = adj[m * W + w];
                while (up) {
                    int y = (w << 5) + __ffs(up) - 1;
                    up &= up - 1u;
                    add_pair(y, G[e++]);
                }
                unsigned dn = adjT[m * W + w];
                while (dn) {
                    int x = (w << 5) + __ffs(dn) - 1;
                    dn &= dn - 1u;
                    add_pair(x, G[rowoff[x] + rank(x, m)]);
                }
            }
        } else {
            for (int y = 0; y < M; y++) {
                if (y == m) continue;
                add_pair(y, G[y > m ? tri_index(m, y) : tri_index(y, m)]);
            }
        }
        double f0 = fxs.get(), f1 = fys.get(), f2 = fzs.get();
        int g = sidx[m];
        if (f0 != 0.0) atomicAdd(A.fs + g, f0);
        if (f1 != 0.0) atomicAdd(A.fs + n + g, f1);
        if (f2 != 0.0) atomicAdd(A.fs + 2 * n + g, f2);
    }

    unsigned long long cand = 0;
    if (tid == 0) cand = unit_candidates<TRAV, S>(s_beg);
    unit_reduce_store<8>(esum.get(), wsum.get(), (unsigned long long)nint, 1.0, cand, A.unit_ew,
                         A.unit_cnt, u, s_red, s_redn);
}

}  // namespace atm3
