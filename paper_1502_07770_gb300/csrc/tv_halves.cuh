// One thread per chain half, for any row or column chain policy of tv_dp.cuh.
//
// Algorithm 2 may take any node as the root: chain k is rooted at node mid = n/2;
// lane l < 16 of a warp runs the forward pass of the warp's chain l over nodes
// 0..mid-1, lane l + 16 over nodes n-1..mid+1 (the same update: the pairwise terms are
// symmetric). Each half ends with the message into the root; the left lane solves
//     z - c_mid + m_L(z) + m_R(z) = 0
// by one merged walk over both halves' breakpoint sequences (the partner's ring is in
// the same shared memory), and both lanes clip their halves outwards from x_mid
// (Algorithm 2, backward). Twice the warps of one thread per chain, each with half the
// steps.
//
// Beyond the chain_batch_kernel interface a policy gives WI, the index of its edge
// weight input (-1: none staged); a right-half lane stages weight i-1 with node i (the
// edge towards the root). unary() is called with n = i + 2, because every node of a
// half has an edge towards the root. Policies with bind_warp() bind 16 chains per warp
// (bind_warp(w * 16)); rec_slot() gives the warp's records: 32 lanes x ceil(len / 2).
// A chain whose half outgrows the ring is solved whole by its left lane from the
// workspace (two-ended array of Sec. 4.1, records at stride 16).
#pragma once
#include "tv_coop.cuh"
#include "tv_dp.cuh"

namespace tvk {

constexpr int HW = WARP / 2;  // chains per warp

template <class P, int RING>
struct alignas(16) HalfSmem {
    union {
        struct {
            float in[P::NIN][2][WARP * RP];
            float2 ring[RING][WARP];
        } f;
        struct {
            float2 rec[2][CH][WARP];
            float crec[P::CREC ? 2 : 1][P::CREC ? CH : 1][WARP];
            float out[WARP * RP];
        } b;
    } u;
    long long start[WARP];
    int n[WARP];
    int cnt[WARP];   // steps of each lane's half
};

// node of step j of a half (left: j; right: n-1-j)
__device__ __forceinline__ int half_node(int lane, int n, int j)
{
    return lane < HW ? j : n - 1 - j;
}

// Row inputs in bit a of `vmask` (16-byte aligned rows of a multiple of 4 nodes) are
// copied by each lane for its own half: the chunk's CH nodes as CH/4 16-byte pieces, in
// memory order. A left half's steps ascend with the nodes, so step jj of the chunk sits at
// tile position jj; a right half's descend, so step jj sits at CH-1-jj. Pieces that would
// leave the chain are copied node by node. With `vw` the edge weights are copied per lane
// too (see the weights branch). Otherwise an input is copied 4 bytes at a time, 8 lanes per
// row, for every lane's row (k is this lane's chain, wc0 the warp's first).
template <class P, int RING>
__device__ __forceinline__ void half_fill(const P &p, HalfSmem<P, RING> *sm, int b, int chunk,
                                          int lane, long long wc0, unsigned vmask, bool vw,
                                          long long k, long long start, int n, int cnt)
{
#pragma unroll
    for (int a = 0; a < P::NIN; ++a) {
        const float *src = p.in_ptr(a);
        if (src == nullptr) continue;
        float *tile = sm->u.f.in[a][b];
        if (!P::COLS && a == P::WI && vw) {
            // edge weights, each lane for its own half: a left half's weight of step jj is
            // node jj's (tile position jj); a right half's is node n-2-j's, so the chunk's
            // eight lie in the 12-float window from n-12-chunk*CH, step jj at 10-jj
            if (chunk * CH < cnt) {
                const float *row = src + p.in_off(a, k, start);
                const int lim = p.in_lim(a, n);
                const bool lft = lane < HW;
                const int w0 = lft ? chunk * CH : n - 12 - chunk * CH;
#pragma unroll
                for (int h = 0; h < 3; ++h) {
                    if (lft && h == 2) break;
                    const int lo = w0 + 4 * h;
                    if (lo >= 0 && lo + 3 < lim && (((uintptr_t)(row + lo)) & 15) == 0) {
                        cp_async16(&tile[lane * RP + 4 * h], row + lo);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (lo + e >= 0 && lo + e < lim)
                                cp_async4(&tile[lane * RP + 4 * h + e], row + lo + e);
                    }
                }
            }
            continue;
        }
        if (!P::COLS && ((vmask >> a) & 1u)) {
            if (chunk * CH < cnt) {
                const float *row = src + p.in_off(a, k, start);
                const int lim = p.in_lim(a, n);
#pragma unroll
                for (int h = 0; h < CH / 4; ++h) {
                    const int lo = lane < HW ? chunk * CH + 4 * h : n - CH - chunk * CH + 4 * h;
                    if (lo >= 0 && lo + 3 < lim) {
                        cp_async16(&tile[lane * RP + 4 * h], row + lo);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (lo + e >= 0 && lo + e < lim)
                                cp_async4(&tile[lane * RP + 4 * h + e], row + lo + e);
                    }
                }
            }
            continue;
        }
        if constexpr (P::COLS) {
            // node j of every lane's column: 16 left lanes and 16 right lanes each read
            // 16 neighbouring columns of one node row
            const long long kb = col_base_of(p, wc0);
            const long long ld = p.in_ld(a);
#pragma unroll 4
            for (int jj = 0; jj < CH; ++jj) {
                const int j = chunk * CH + jj;
                if (j < sm->cnt[lane]) {
                    const int i = half_node(lane, sm->n[lane], j);
                    const int ii = (a == P::WI && lane >= HW) ? i - 1 : i;
                    cp_async4(&tile[lane * RP + jj], src + (long long)ii * ld + kb + (lane & (HW - 1)));
                }
            }
        } else {
            // 8 consecutive nodes of one lane's row per 8 lanes
#pragma unroll 4
            for (int u = 0; u < CH; ++u) {
                const int t = u * WARP + lane;
                const int lt = t / CH, jj = t % CH;
                const int j = chunk * CH + jj;
                if (j < sm->cnt[lt]) {
                    const int i = half_node(lt, sm->n[lt], j);
                    const int ii = (a == P::WI && lt >= HW) ? i - 1 : i;
                    const long long kt = wc0 + (lt & (HW - 1));  // the chain of row lt
                    cp_async4(&tile[lt * RP + jj], src + p.in_off(a, kt, sm->start[lt]) + ii);
                }
            }
        }
    }
}

// The whole chain by one thread, from node 0 (overflow path). Records (and c records)
// at stride 16 from rec16. Policies that record c_i give it by c_direct() here.
template <class P>
__device__ void half_fallback(const P &p, long long k, long long start, int n, float2 *spill,
                              float2 *rec16, float *crec16)
{
    LinearStore S{spill};
    DPState d;
    float lm = 0.f, hp = 0.f, c = 0.f, w = 0.f;
    float xlast = 0.f;
    for (int i = 0; i < n; ++i) {
        p.unary_direct(i, n, k, start, c, w);
        if constexpr (P::CREC) {
            c = p.c_direct(i, k, start);
            crec16[(long long)i * HW] = c;
        }
        if (i == 0) {
            if (n == 1) {
                xlast = c;
                break;
            }
            dp_first(d, S, n, c, w, lm, hp);
        } else {
            dp_step(d, S, 2 * n + 2, c, w, (float)(i + 1), lm, hp);
        }
        if (i == n - 1) xlast = 0.5f * (lm + hp);
        else rec16[(long long)i * HW] = make_float2(lm, hp);
    }
    float xv = xlast;
    for (int i = n - 1; i >= 0; --i) {
        float cc = 0.f;
        if constexpr (P::CREC) cc = crec16[(long long)i * HW];
        if (i < n - 1) {
            const float2 r = rec16[(long long)i * HW];
            xv = clip_to(xv, r.x, r.y);
        }
        p.emit_direct(i, k, start, xv, cc);
    }
}

// Root of z - c + m_L(z) + m_R(z): each message is -w left of its first breakpoint,
// +w right of its last, with slope s_p + abar right of breakpoint p (abar = the half's
// node count); an empty half contributes 0. St: a store with ld(index) (ring or linear);
// max_steps bounds the walk (both messages hold at most max_steps - 4 breakpoints).
template <class St>
__device__ __forceinline__ float half_root(const St &SL, int FL, int BL, float aL, float wL,
                                           const St &SR, int FR, int BR, float aR, float wR,
                                           float c, int max_steps)
{
    const bool hasL = BL >= FL, hasR = BR >= FR;
    if (!hasL) wL = 0.f;
    if (!hasR) wR = 0.f;
    int pL = FL, pR = FR;
    float2 eL = hasL ? SL.ld(pL) : make_float2(INFINITY, 0.f);
    float2 eR = hasR ? SR.ld(pR) : make_float2(INFINITY, 0.f);
    float zc = fminf(eL.x, eR.x);
    if (!(zc < INFINITY)) return c;  // no message at all
    float hc = zc - c - wL - wR;      // h at the first breakpoint (slope 1 to its left)
    float slope = 1.f;                // slope of h on the segment ending at zc
    for (int it = 0; it < max_steps; ++it) {
        if (hc >= 0.f) return zc - hc / slope;
        // pass the breakpoint(s) at zc; the slopes right of it come from the last
        // breakpoint passed in each half
        if (hasL && pL <= BL && eL.x == zc) {
            ++pL;
            eL = pL <= BL ? SL.ld(pL) : make_float2(INFINITY, 0.f);
        }
        if (hasR && pR <= BR && eR.x == zc) {
            ++pR;
            eR = pR <= BR ? SR.ld(pR) : make_float2(INFINITY, 0.f);
        }
        const float gL = (hasL && pL > FL) ? SL.ld(pL - 1).y + aL : 0.f;
        const float gR = (hasR && pR > FR) ? SR.ld(pR - 1).y + aR : 0.f;
        slope = 1.f + gL + gR;
        const float zn = fminf(eL.x, eR.x);
        if (!(zn < INFINITY)) return zc - hc / slope;
        hc = fmaf(slope, zn - zc, hc);
        zc = zn;
    }
    return zc - hc / slope;  // not reached: at most 2 (RING + 1) breakpoints
}

template <class P, int RING>
__global__ void __launch_bounds__(128) chain_halves_kernel(P p_in, float2 *rec, float *crec,
                                                           float2 *spill, WsHeader *hdr,
                                                           int halfmax)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    P p = p_in;
    if (!p.resolve()) return;
    const int lane = threadIdx.x & (WARP - 1);
    const int warp = threadIdx.x / WARP;
    const int wpb = blockDim.x / WARP;
    HalfSmem<P, RING> *sm = reinterpret_cast<HalfSmem<P, RING> *>(smem_raw) + warp;
    const long long wg = (long long)blockIdx.x * wpb + warp;
    const long long wc0 = wg * HW;
    const long long k = wc0 + (lane & (HW - 1));
    const bool left = lane < HW;
    if constexpr (has_bind<P>::value) {
        if (wc0 >= p.num_chains() || !p.bind_warp(wc0)) {
            p.finish_empty();
            return;
        }
    }
    long long start = 0;
    int n = 0;
    if (k < p.num_chains()) {
        if (!p.chain(k, start, n)) {
            if (left) atomicOr(&hdr->status, ERR_BAD_CHAIN);
            n = 0;
        }
    }
    const int mid = n >> 1;
    const int cnt = n == 0 ? 0 : (left ? mid : n - 1 - mid);  // update steps of this half
    // row inputs and outputs moved 16 bytes at a time by each lane for its own half
    // (edge weights excepted: a right half reads them one node off the 4-node grid)
    unsigned vmask = 0;
    bool vout = false, vw = false;
    if constexpr (!P::COLS) {
#pragma unroll
        for (int a = 0; a < P::NIN; ++a)
            if (a != P::WI && p.in_vec(a)) vmask |= 1u << a;
        vout = p.out_vec();
        if constexpr (P::WI >= 0) vw = p.in_vec(P::WI);  // weights in per-lane windows
    }
    // the staging layouts are shared across the warp's lanes: keep them warp-uniform
    vmask = __reduce_and_sync(FULL, vmask);
    vout = __all_sync(FULL, vout);
    vw = __all_sync(FULL, vw);
    sm->start[lane] = start;
    sm->n[lane] = n;
    sm->cnt[lane] = cnt;
    int cmax = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cmax = max(cmax, __shfl_xor_sync(FULL, cmax, o));
    __syncwarp();
    long long slot = wg * (long long)halfmax * WARP;
    if constexpr (has_rec_slot<P>::value) slot = p.rec_slot(wg, halfmax);
    float2 *rec_w = rec + slot;
    float *crec_w = P::CREC ? crec + slot : nullptr;
    RingStore<RING> S{(unsigned)__cvta_generic_to_shared(&sm->u.f.ring[0][lane])};
    DPState d;
    d.F = 0;
    d.B = -1;
    d.w_prev = 0.f;
    typename P::Acc acc;
    p.acc_init(acc);
    bool alive = true;
    const int nchunks = (cmax + CH - 1) / CH;

    // ---------------- forward pass over each half ----------------
    if (nchunks > 0) half_fill(p, sm, 0, 0, lane, wc0, vmask, vw, k, start, n, cnt);
    cp_async_commit();
    int b = 0;
    for (int ch = 0; ch < nchunks; ++ch) {
        if (ch + 1 < nchunks)
            half_fill(p, sm, b ^ 1, ch + 1, lane, wc0, vmask, vw, k, start, n, cnt);
        cp_async_commit();
        cp_async_wait<1>();
        __syncwarp();
#pragma unroll 1
        for (int j4 = 0; j4 < CH; j4 += 4) {
            float4 q[P::NIN];
            const unsigned rv = left ? 0u : vmask;  // inputs whose steps run backwards in the tile
            // a right half's windowed weights: steps j4..j4+3 at positions 10-j4 .. 7-j4
            const bool rw = !left && vw;
            float4 qw = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int a = 0; a < P::NIN; ++a) {
                const int pos = (a == P::WI && rw) ? CH - j4 : (((rv >> a) & 1u) ? CH - 4 - j4 : j4);
                q[a] = *reinterpret_cast<const float4 *>(&sm->u.f.in[a][b][lane * RP + pos]);
                if (a == P::WI && rw)
                    qw = *reinterpret_cast<const float4 *>(&sm->u.f.in[a][b][lane * RP + CH - 4 - j4]);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = ch * CH + j4 + e;
                if (j < cnt && alive) {
                    float v[P::NIN];
#pragma unroll
                    for (int a = 0; a < P::NIN; ++a) {
                        if (a == P::WI && rw) v[a] = e < 3 ? pick4(q[a], 2 - e) : qw.w;
                        else v[a] = ((rv >> a) & 1u) ? pick4(q[a], 3 - e) : pick4(q[a], e);
                    }
                    const int i = half_node(lane, n, j);
                    float c, w;
                    p.unary(v, 0.f, j, i, i + 2, k, c, w, acc);
                    if constexpr (P::CREC) crec_w[(long long)j * WARP + lane] = c;
                    float lm, hp;
                    if (j == 0) dp_first(d, S, 0, c, w, lm, hp);
                    else alive = dp_step(d, S, RING, c, w, (float)(j + 1), lm, hp);
                    if (alive) rec_w[(long long)j * WARP + lane] = make_float2(lm, hp);
                }
            }
        }
        __syncwarp();
        b ^= 1;
    }
    cp_async_wait<0>();
    __syncwarp();

    // ---------------- root ----------------
    const int FR = __shfl_down_sync(FULL, d.F, HW), BR = __shfl_down_sync(FULL, d.B, HW);
    const float wR = __shfl_down_sync(FULL, d.w_prev, HW);
    const int cntR = __shfl_down_sync(FULL, cnt, HW);
    const bool aliveR = __shfl_down_sync(FULL, (int)alive, HW) != 0;
    const bool ok = __shfl_sync(FULL, (int)(alive && aliveR), lane & (HW - 1)) != 0;
    float xroot = 0.f;
    if (left && n > 0 && ok) {
        // c of the root node, from global memory
        float c_root, w_unused;
        p.unary_direct(mid, n, k, start, c_root, w_unused);
        if constexpr (P::CREC) c_root = p.c_direct(mid, k, start);
        const RingStore<RING> SR{S.base + HW * 8};  // lane + 16's ring
        xroot = half_root(S, cnt > 0 ? d.F : 0, cnt > 0 ? d.B : -1, (float)cnt, d.w_prev, SR,
                          cntR > 0 ? FR : 0, cntR > 0 ? BR : -1, (float)cntR, wR, c_root,
                          2 * RING + 4);
        p.emit_direct(mid, k, start, xroot, c_root);
    }
    xroot = __shfl_sync(FULL, xroot, lane & (HW - 1));
    __threadfence_block();
    __syncwarp();

    // ---------------- backward pass, outwards from the root ----------------
    const int cnt_eff = ok ? cnt : 0;
    sm->cnt[lane] = cnt_eff;
    float xv = xroot;
    auto load_recs = [&](int buf, int ch) {
#pragma unroll 4
        for (int u = 0; u < CH; ++u) {
            const int j = ch * CH + u;
            if (j < cnt_eff) {
                cp_async8(&sm->u.b.rec[buf][u][lane], rec_w + (long long)j * WARP + lane);
                if constexpr (P::CREC)
                    cp_async4(&sm->u.b.crec[buf][u][lane], crec_w + (long long)j * WARP + lane);
            }
        }
    };
    b = 0;
    if (nchunks > 0) load_recs(0, nchunks - 1);
    cp_async_commit();
    for (int ch = nchunks - 1; ch >= 0; --ch) {
        if (ch > 0) load_recs(b ^ 1, ch - 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncwarp();
        bool stored = false;
        if constexpr (!P::COLS) {
            if (vout) {
                // each lane stores its own half: 4 steps in registers, then the group's 4
                // nodes (lowest first) with one 16-byte store, or node by node when the
                // group holds steps beyond the half
#pragma unroll
                for (int g = CH / 4 - 1; g >= 0; --g) {
                    float xs[4];
#pragma unroll
                    for (int e = 3; e >= 0; --e) {
                        const int jj = 4 * g + e;
                        xs[e] = 0.f;
                        if (ch * CH + jj < cnt_eff) {
                            const float2 r = sm->u.b.rec[b][jj][lane];
                            xv = clip_to(xv, r.x, r.y);
                            xs[e] = xv;
                        }
                    }
                    const int j0 = ch * CH + 4 * g;
                    const int lo = left ? j0 : n - 4 - j0;
#pragma unroll
                    for (int o = 0; o < P::NOUT; ++o) {
                        float *dst = p.out_ptr(o) + p.out_off(o, k, start);
                        if (j0 + 3 < cnt_eff) {
                            *reinterpret_cast<float4 *>(dst + lo) =
                                left ? make_float4(xs[0], xs[1], xs[2], xs[3])
                                     : make_float4(xs[3], xs[2], xs[1], xs[0]);
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (j0 + e < cnt_eff) dst[left ? lo + e : lo + 3 - e] = xs[e];
                        }
                    }
                }
                stored = true;
            }
        }
        if (!stored) {
#pragma unroll 4
            for (int jj = CH - 1; jj >= 0; --jj) {
                const int j = ch * CH + jj;
                if (j < cnt_eff) {
                    const float2 r = sm->u.b.rec[b][jj][lane];
                    xv = clip_to(xv, r.x, r.y);
                    if constexpr (P::COLS) {
                        float cc = 0.f;
                        if constexpr (P::CREC) cc = sm->u.b.crec[b][jj][lane];
                        p.emit_cols(half_node(lane, n, j), k, xv, cc);
                    } else {
                        sm->u.b.out[lane * RP + jj] = xv;
                    }
                }
            }
            if constexpr (!P::COLS) {
                __syncwarp();
#pragma unroll
                for (int o = 0; o < P::NOUT; ++o) {
                    float *dst = p.out_ptr(o);
#pragma unroll 4
                    for (int u = 0; u < CH; ++u) {
                        const int t = u * WARP + lane;
                        const int lt = t / CH, jj = t % CH;
                        const int j = ch * CH + jj;
                        if (j < sm->cnt[lt])
                            dst[p.out_off(o, wc0 + (lt & (HW - 1)), sm->start[lt]) +
                                half_node(lt, sm->n[lt], j)] = sm->u.b.out[lt * RP + jj];
                    }
                }
            }
        }
        __syncwarp();
        b ^= 1;
    }
    cp_async_wait<0>();
    if (left && n > 0 && !ok) {
        atomicAdd(&hdr->overflowed, 1ull);
        float *c16 = P::CREC ? crec_w + lane : nullptr;
        half_fallback(p, k, start, n, spill + p.spill_off(k, start), rec_w + lane, c16);
    }
    p.finish(acc);
}

}  // namespace tvk
