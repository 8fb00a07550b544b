// Warp-cooperative chain dynamic program: one warp per chain.
//
// The same messages as tv_dp.cuh (Algorithm 2 specialised to quadratic unaries,
// Sec. 4.1), laid out for latency: the breakpoints of the chain's current message
// live in registers, breakpoint k in lane k (at most 32), each with the message's
// value there. At node i:
//   * every lane adds lambda_k - c_i to its value (transformation (a));
//   * two ballots count the breakpoints removed on each side (values < -w_i from
//     the left, > w_i from the right among those kept);
//   * every lane computes where the piece to its right crosses -w_i and +w_i, and
//     the lanes next to the removed runs broadcast lambda^- and lambda^+;
//   * one shuffle shifts the kept breakpoints into place between the two new ones.
// The records lambda^-_i, lambda^+_i go to shared memory (global memory for long
// chains). The backward clips x_i = clip(x_{i+1}, lambda^-_i, lambda^+_i) are
// composed 32 nodes at a time by a warp suffix scan: clip_[a1,b1] o clip_[a2,b2]
// = clip_[clip(a2,a1,b1), clip(b2,a1,b1)], an associative operation.
//
// A message of more than 32 breakpoints is finished from global memory by lane 0
// with the sequential update of tv_dp.cuh (two-ended array of 2n+2 entries).
#pragma once
#include <type_traits>

#include "tv_dp.cuh"

namespace tvk {

constexpr unsigned FULL = 0xffffffffu;

// Composition of the backward clips of nodes j..31 of a 32-node block, applied
// to x_next (the value of the node after the block): lane j returns x of its node.
__device__ __forceinline__ float clip_suffix(float lo, float hi, float x_next, int lane, int valid)
{
    // invalid lanes (beyond the chain) are the identity clip
    if (lane >= valid) {
        lo = -INFINITY;
        hi = INFINITY;
    }
#pragma unroll
    for (int o = 1; o < WARP; o <<= 1) {
        const float lo2 = __shfl_down_sync(FULL, lo, o);
        const float hi2 = __shfl_down_sync(FULL, hi, o);
        if (lane + o < WARP) {
            // this lane's clip applied after the clip of lanes lane+o.. (inner)
            const float nlo = clip_to(lo2, lo, hi);
            const float nhi = clip_to(hi2, lo, hi);
            lo = nlo;
            hi = nhi;
        }
    }
    return clip_to(x_next, lo, hi);
}

// Overflow path of the cooperative kernel: lane 0 re-solves its chain with the
// sequential update of tv_dp.cuh, the message in a two-ended array of 2n+2
// entries in global memory (Sec. 4.1) and the records in rec[0..n) (global).
template <class P>
__device__ void solve_chain_global_lane0(const P &p, long long k, long long start, int n,
                                         float2 *spill, float2 *rec, const float *crec)
{
    LinearStore S{spill};
    DPState d;
    float lm = 0.f, hp = 0.f, c, w;
    float xlast = 0.f;
    for (int i = 0; i < n; ++i) {
        p.unary_direct(i, n, k, start, c, w);
        if constexpr (P::CREC) c = crec[i];
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
        else rec[i] = make_float2(lm, hp);
    }
    float xv = xlast;
    for (int i = n - 1; i >= 0; --i) {
        float cc = 0.f;
        if constexpr (P::CREC) cc = crec[i];
        if (i < n - 1) {
            const float2 r = rec[i];
            xv = clip_to(xv, r.x, r.y);
        }
        p.emit_direct(i, k, start, xv, cc);
    }
}

// Shared memory of one warp: `nodes` records lambda^-_i, lambda^+_i, then (if the
// policy records c_i) `nodes` floats.
template <class P>
__host__ __device__ constexpr size_t coop_smem_per_warp(int nodes)
{
    return (size_t)nodes * (sizeof(float2) + (P::CREC ? sizeof(float) : 0));
}

// The warp-cooperative message update of one node. Lane k of a group of G lanes
// (the warp, G = 32, or a 16-lane half) holds breakpoint lambda_k of the message
// m_{i-1,i} (a derivative: continuous, increasing, piecewise linear, -w_{i-1} left
// of the first breakpoint and +w_{i-1} right of the last), the message's value V_k
// there and its slope T_k on the piece to the right (an integer, the number of
// nodes fused on that piece; 0 right of the last breakpoint). Transformation (a),
// m^_i = m_{i-1,i} + z - c_i, is the lane-local v_k = V_k + lambda_k - c_i with
// slope S_k = T_k + 1; the left scan removes the prefix with v < -w_i, the right
// scan the suffix with v > w_i among the rest, and lambda^-, lambda^+ are where the
// piece right of the last removed (resp. last kept) breakpoint crosses -w_i, +w_i:
// lambda_k + (+-w_i - v_k) / S_k, clamped to the piece. The quotient's reciprocal
// depends only on the stored slope, so it is off the step's critical path, and the
// exact integer slopes keep the crossings precise in FP32.
// A new message of more than G breakpoints sets `ovf` (sticky); the state is then
// meaningless and the caller re-solves the chain on the overflow path.
__device__ __forceinline__ float seg_frac(float num, float den)
{
    // fraction along a segment, clamped to [0, 1] (0 for a zero-length segment)
    return fminf(fmaxf(__fdividef(num, den), 0.f), 1.f);
}

// General form (Sec. 4, Sec. 4.1): unary a_i x^2/2 - b_i x, pairwise slopes w^-_i <= w^+_i.
// m^_i = m_{i-1,i} + a_i z - b_i; the message is clipped to [w^-_i, w^+_i]; the end pieces
// of m^_i have slope a_i. `wl_prev` is w^-_{i-1} (the message's value left of its first
// breakpoint). TV-l2 is a_i = 1, b_i = c_i, w^-_i = -w_i, w^+_i = w_i.
// ALWAYS: every lane of the group updates (compile-time `active`).
template <int G, bool ALWAYS = false>
__device__ __forceinline__ void coop_update_g(float &lam, float &V, float &T, int &size,
                                              float &wl_prev, float ai, float bi,
                                              float wl, float wh, int sl, int seg_shift,
                                              bool active, bool &ovf, float &lm, float &hp)
{
    const bool valid = sl < size;
    const bool last = sl == size - 1;
    const float S = T + ai;                    // slope of m^_i right of this breakpoint
    const float v = fmaf(ai, lam, V) - bi;     // m^_i at this breakpoint
    const float lam_n = __shfl_down_sync(FULL, lam, 1, G);
    const float rS = __fdividef(1.f, S);  // one reciprocal for both crossings
    float candL = fmaxf(fmaf(wl - v, rS, lam), lam);
    float candR = fmaxf(fmaf(wh - v, rS, lam), lam);
    if (!last) {
        candL = fminf(candL, lam_n);
        candR = fminf(candR, lam_n);
    }
    // first lane with v >= w^- and last lane with v <= w^+: one vote each, then the
    // lowest / highest set bit of this segment's bits
    unsigned bge = __ballot_sync(FULL, valid && v >= wl);
    unsigned ble = __ballot_sync(FULL, valid && v <= wh);
    // (trailing zeros of an empty vote are 32, so ell is then size. Bits of the segment
    // above only count when none of this segment's is set, and then ell = size <= G too;
    // the highest set bit is taken among this segment's bits, -1 - seg_shift if none,
    // which keep_last = max(kl, ell - 1) treats as -1.)
    if constexpr (G != WARP) bge >>= seg_shift;
    const int ell = min(__clz(__brev(bge)), size);
    int kl;
    if constexpr (G != WARP) kl = 31 - seg_shift - __clz(ble & (((1u << G) - 1u) << seg_shift));
    else kl = 31 - __clz(ble);
    const int keep_last = kl > ell - 1 ? kl : ell - 1;  // last kept breakpoint (-1: none)
    const int K = keep_last - ell + 1;
    ovf = ovf || ((ALWAYS || active) && K + 2 > G);
    // lambda^- on the piece right of the last breakpoint removed on the left,
    // lambda^+ on the piece right of the last one kept; with none, on the left end
    // piece, where m^_i = w^-_{i-1} + a_i z - b_i
    // source lanes are taken modulo the segment width by the shuffles themselves
    const float gl = __shfl_sync(FULL, candL, ell - 1, G);
    const float gr = __shfl_sync(FULL, candR, keep_last, G);
    lm = (ell == 0) ? (bi + wl - wl_prev) / ai : gl;
    hp = (keep_last < 0) ? (bi + wh - wl_prev) / ai : gr;
    // new message m_{i,i+1}: lambda^- (value w^-_i, the slope of m^_i there), the kept
    // breakpoints with their values and slopes, lambda^+ (value w^+_i, flat beyond);
    // lane 0's source is breakpoint ell-1, so its nS is the slope right of lambda^-
    const int src = sl - 1 + ell;
    const float nl = __shfl_sync(FULL, lam, src, G);
    const float nv = __shfl_sync(FULL, v, src, G);
    const float nS = __shfl_sync(FULL, S, src, G);
    if (ALWAYS || active) {
        lam = (sl == 0) ? lm : ((sl == K + 1) ? hp : nl);
        V = (sl == 0) ? wl : ((sl == K + 1) ? wh : nv);
        T = (sl == 0 && ell == 0) ? ai : ((sl == K + 1) ? 0.f : nS);
        size = K + 2;
        wl_prev = wl;
    }
}

// TV-l2 form: a_i = 1, b_i = c_i, [w^-_i, w^+_i] = [-w_i, w_i]; `w_prev` is w_{i-1}.
template <int G, bool ALWAYS = false>
__device__ __forceinline__ void coop_update(float &lam, float &V, float &T, int &size,
                                            float &w_prev, float ci, float wi,
                                            int sl, int seg_shift, bool active, bool &ovf,
                                            float &lm, float &hp)
{
    float wl_prev = -w_prev;
    coop_update_g<G, ALWAYS>(lam, V, T, size, wl_prev, 1.f, ci, -wi, wi, sl, seg_shift,
                             active, ovf, lm, hp);
    if (ALWAYS || active) w_prev = wi;
}

// Start of a message at the first node of a walk: m_{0,1} = clip(z - c_0, -w_0, w_0).
__device__ __forceinline__ void coop_first(float &lam, float &V, float &T, int &size,
                                           float &w_prev, float ci, float wi, int sl, float &lm,
                                           float &hp)
{
    lm = ci - wi;
    hp = ci + wi;
    lam = (sl == 0) ? lm : hp;
    V = (sl == 0) ? -wi : wi;
    T = (sl == 0) ? 1.f : 0.f;
    size = 2;
    w_prev = wi;
}

// Policy interface (P):
//   static constexpr int SMEM_NODES   records kept in shared memory per warp
//   static constexpr bool CREC        the epilogue needs c_i
//   struct Raw, struct Acc
//   resolve(), num_chains(), max_len(), chain(k, &start, &n)
//   fetch(k, start, n, i, Raw&)              loads of node i (lane-parallel, i may be >= n)
//   unary(k, start, n, i, const Raw&, Raw* prev, &c, &w, Acc&)   c_i, w_i of node i
//   emit(k, start, i, xhat, c)               output of node i
//   unary_direct(i, n, k, start, &c, &w), emit_direct(i, k, start, xhat, c)   overflow path
//   spill_off(k, start), acc_init(Acc&), finish(Acc&, lane), finish_empty()

// One chain (index k, first node `start`, n nodes) solved by the calling warp:
// forward message pass, records, backward clips, output through the policy.
// Records stay in sm_rec/sm_crec (smem_nodes entries) when the chain fits, else in
// rec_g/crec_g at slot k * max_len; `spill` is the chain's overflow reserve base.
template <class P>
__device__ void coop_solve_chain(const P &p, typename P::Acc &acc, long long k, long long start,
                                 int n, int lane, float2 *sm_rec, float *sm_crec, int smem_nodes,
                                 float2 *rec_g, float *crec_g, float2 *spill, WsHeader *hdr)
{
    const int max_len = p.max_len();
    // records: shared memory when the chain fits, else this chain's global slot
    const bool in_smem = n <= smem_nodes;
    float2 *recp = in_smem ? sm_rec : rec_g + k * (long long)max_len;
    float *crecp = nullptr;
    if constexpr (P::CREC) crecp = in_smem ? sm_crec : crec_g + k * (long long)max_len;

    float lam = 0.f, V = 0.f, T = 0.f, w_prev = 0.f;
    int size = 0;
    bool ok = true, ovf = false;
    float xlast = 0.f;

    typename P::Raw raw, raw_next{};
    p.fetch(k, start, n, lane, raw);
    const int nblocks = (n + WARP - 1) / WARP;
    for (int blk = 0; blk < nblocks; ++blk) {
        const int base = blk * WARP;
        if (blk + 1 < nblocks) p.fetch(k, start, n, base + WARP + lane, raw_next);
        float cv, wv;
        p.unary(k, start, n, base + lane, raw, cv, wv, acc);  // lane-parallel
        if constexpr (P::CREC) {
            if (base + lane < n) crecp[base + lane] = cv;
        }
        const int cnt = min(WARP, n - base);
        if (ok) {
            for (int j = 0; j < cnt; ++j) {
                const int i = base + j;
                const float ci = __shfl_sync(FULL, cv, j);
                const float wi = (i < n - 1) ? __shfl_sync(FULL, wv, j) : 0.f;
                float lmv, hpv;
                if (i == 0) {
                    if (n == 1) {
                        xlast = ci;
                        break;
                    }
                    coop_first(lam, V, T, size, w_prev, ci, wi, lane, lmv, hpv);
                } else {
                    coop_update<WARP>(lam, V, T, size, w_prev, ci, wi, lane, 0, true, ovf,
                                      lmv, hpv);
                }
                if (i == n - 1) xlast = 0.5f * (lmv + hpv);
                else if (lane == 0) recp[i] = make_float2(lmv, hpv);
            }
            ok = !ovf;  // warp-uniform: the group is the whole warp
        }
        raw = raw_next;
    }
    __syncwarp();

    if (ok) {
        // backward: 32 nodes at a time from the end, composing clips
        float x_next = xlast;
        for (int blk = nblocks - 1; blk >= 0; --blk) {
            const int base = blk * WARP;
            const int i = base + lane;
            float lo = -INFINITY, hi = INFINITY;
            if (i < n - 1) {
                const float2 r = recp[i];
                lo = r.x;
                hi = r.y;
            }
            const int valid = min(WARP, n - base);
            // node n-1 has no clip: it is x_last itself (identity clip there)
            float xv = clip_suffix(lo, hi, x_next, lane, valid);
            float cc = 0.f;
            if constexpr (P::CREC) {
                if (i < n) cc = crecp[i];
            }
            if (i < n) p.emit(k, start, i, xv, cc);
            // the first node of this block feeds the block before it
            x_next = __shfl_sync(FULL, xv, 0);
        }
    } else {
        if (lane == 0) {
            atomicAdd(&hdr->overflowed, 1ull);
            solve_chain_global_lane0(p, k, start, n, spill, rec_g + k * (long long)max_len,
                                     crecp);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------
// Two warps per chain. A chain is a tree, and Algorithm 2 may take any node as the
// root: with the middle node s = n/2 as root, the messages into s from the left
// (nodes 0..s-1, the usual forward pass) and from the right (nodes n-1..s+1, the same
// pass on the reversed chain) are independent, so two warps compute them at once and
// the sequential depth halves. x_s minimises the unary of s plus both messages: the
// root of h(z) = z - c_s + mL'(z) + mR'(z), a continuous increasing piecewise-linear
// function whose kinks are the two messages' breakpoints. Each warp then runs its
// backward clips outward from s: x_i = clip(x_{i+1}, lambda^-_i, lambda^+_i) on the
// left, x_i = clip(x_{i-1}, lambda^-_i, lambda^+_i) on the right (the records of the
// reversed pass).

// Composition of the clips of lanes 0..j applied to x_prev (the value of the node
// before the block): lane j returns x of its node (the right warp's backward pass).
__device__ __forceinline__ float clip_prefix(float lo, float hi, float x_prev, int lane, int valid)
{
    if (lane >= valid) {
        lo = -INFINITY;
        hi = INFINITY;
    }
#pragma unroll
    for (int o = 1; o < WARP; o <<= 1) {
        const float lo2 = __shfl_up_sync(FULL, lo, o);
        const float hi2 = __shfl_up_sync(FULL, hi, o);
        if (lane >= o) {
            // this lane's clip applied after the clips of the lanes below (inner)
            const float nlo = clip_to(lo2, lo, hi);
            const float nhi = clip_to(hi2, lo, hi);
            lo = nlo;
            hi = nhi;
        }
    }
    return clip_to(x_prev, lo, hi);
}

// A message (derivative) stored by a warp for its partner: breakpoints ascending,
// the message's value at each; constant left of the first and right of the last.
struct PairMsg {
    float lam[WARP];
    float val[WARP];
    int size;
    int ok;
};
struct alignas(16) PairXchg {
    PairMsg m[2];  // [0]: message into s from the left warp, [1]: from the right warp
    float xs;      // x of the root node
};

__device__ __forceinline__ void pair_barrier(int pair)
{
    asm volatile("bar.sync %0, %1;" ::"r"(pair + 1), "r"(2 * WARP) : "memory");
}

// Value at z of a stored message (linear between breakpoints).
__device__ __forceinline__ float msg_eval(const PairMsg &m, float z)
{
    const int size = m.size;
    if (z <= m.lam[0]) return m.val[0];
    if (z >= m.lam[size - 1]) return m.val[size - 1];
    int lo = 0, hi = size - 1;  // invariant: lam[lo] <= z < lam[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (m.lam[mid] <= z) lo = mid;
        else hi = mid;
    }
    const float t = __fdividef(z - m.lam[lo], m.lam[hi] - m.lam[lo]);
    return fmaf(t, m.val[hi] - m.val[lo], m.val[lo]);
}

// Root of h(z) = a z - b + mL'(z) + mR'(z), computed by one warp: lane l evaluates h at
// breakpoint l of each message; the largest point with h <= 0 and the smallest with
// h > 0 are neighbours among all kinks, and h is linear between them.
__device__ __forceinline__ float pair_root(const PairXchg &xc, float a, float b, int lane)
{
    float lo_z = -INFINITY, lo_h = 0.f, hi_z = INFINITY, hi_h = 0.f;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const PairMsg &own = xc.m[side], &oth = xc.m[1 - side];
        if (lane < own.size) {
            const float z = own.lam[lane];
            const float h = fmaf(a, z, -b) + own.val[lane] + msg_eval(oth, z);
            if (h <= 0.f) {
                if (z > lo_z) {
                    lo_z = z;
                    lo_h = h;
                }
            } else if (z < hi_z) {
                hi_z = z;
                hi_h = h;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oz = __shfl_xor_sync(FULL, lo_z, o), oh = __shfl_xor_sync(FULL, lo_h, o);
        if (oz > lo_z) {
            lo_z = oz;
            lo_h = oh;
        }
        const float pz = __shfl_xor_sync(FULL, hi_z, o), ph = __shfl_xor_sync(FULL, hi_h, o);
        if (pz < hi_z) {
            hi_z = pz;
            hi_h = ph;
        }
    }
    const PairMsg &L = xc.m[0], &R = xc.m[1];
    if (lo_z == -INFINITY)  // left of every kink: both messages at their left values
        return fminf((b - L.val[0] - R.val[0]) / a, hi_z);
    if (hi_z == INFINITY)  // right of every kink
        return fmaxf((b - L.val[L.size - 1] - R.val[R.size - 1]) / a, lo_z);
    return fminf(fmaxf(fmaf(-lo_h, __fdividef(hi_z - lo_z, hi_h - lo_h), lo_z), lo_z), hi_z);
}

// Chains shorter than this are solved by the left warp alone.
constexpr int kSplitMinLen = 64;

// One chain solved by a warp pair (role 0: nodes 0..s, role 1: nodes n-1..s+1).
template <class P>
__device__ void coop_solve_chain_split(const P &p, typename P::Acc &acc, long long k,
                                       long long start, int n, int lane, int role, int pair,
                                       PairXchg &xc, float2 *sm_rec, float *sm_crec,
                                       int smem_nodes, float2 *rec_g, float *crec_g,
                                       float2 *spill, WsHeader *hdr)
{
    const int max_len = p.max_len();
    const bool in_smem = n <= smem_nodes;
    float2 *recp = in_smem ? sm_rec : rec_g + k * (long long)max_len;
    float *crecp = nullptr;
    if constexpr (P::CREC) crecp = in_smem ? sm_crec : crec_g + k * (long long)max_len;
    const int s = n / 2;

    float lam = 0.f, V = 0.f, T = 0.f, w_prev = 0.f;
    int size = 0;
    bool ok = true, ovf = false;
    float c_s = 0.f;

    // role 0 walks nodes 0, 1, .., s; role 1 walks n-1, n-2, .., s (node s only for
    // its weight w_s). Position q of the walk is node i(q).
    const int cntw = role == 0 ? s + 1 : n - s;
    auto node = [&](int q) { return role == 0 ? q : n - 1 - q; };
    auto fetch_at = [&](int q, typename P::Raw &r) {
        p.fetch(k, start, n, q < cntw ? node(q) : n, r);
    };
    typename P::Raw raw, raw_next{};
    fetch_at(lane, raw);
    const int nblocks = (cntw + WARP - 1) / WARP;
    for (int blk = 0; blk < nblocks; ++blk) {
        const int base = blk * WARP;
        if (blk + 1 < nblocks) fetch_at(base + WARP + lane, raw_next);
        const int q = base + lane;
        const int i_l = q < cntw ? node(q) : n;
        float cv, wv;
        p.unary(k, start, n, i_l, raw, cv, wv, acc);
        if constexpr (P::CREC) {
            // node s is recorded by the left warp
            if (q < cntw && (role == 0 || i_l != s)) crecp[i_l] = cv;
        }
        // the right warp steps node i with the weight of edge (i-1, i): that of the
        // next position; the block's last lane takes it from the next block
        float wr = 0.f;
        if (role == 1) {
            wr = __shfl_down_sync(FULL, wv, 1);
            float c2, w2;
            p.unary(k, start, n, base + WARP < cntw ? node(base + WARP) : n, raw_next, c2, w2, acc);
            const float w_nb = __shfl_sync(FULL, w2, 0);
            if (lane == WARP - 1) wr = w_nb;
        }
        const int cnt = min(WARP, cntw - base);
        if (ok) {
            for (int j = 0; j < cnt; ++j) {
                const int qq = base + j;
                const float ci = __shfl_sync(FULL, cv, j);
                if (role == 0 && qq == s) {
                    c_s = ci;
                    break;
                }
                if (role == 1 && qq == cntw - 1) break;  // node s: handled by the left warp
                const float wi = __shfl_sync(FULL, role == 0 ? wv : wr, j);
                float lmv, hpv;
                if (qq == 0)
                    coop_first(lam, V, T, size, w_prev, ci, wi, lane, lmv, hpv);
                else
                    coop_update<WARP>(lam, V, T, size, w_prev, ci, wi, lane, 0, true, ovf,
                                      lmv, hpv);
                if (lane == 0) recp[node(qq)] = make_float2(lmv, hpv);
            }
            ok = !ovf;
        }
        raw = raw_next;
    }
    // hand the message into s to the partner
    PairMsg &mine = xc.m[role];
    mine.lam[lane] = lam;
    mine.val[lane] = V;
    if (lane == 0) {
        mine.size = size;
        mine.ok = ok ? 1 : 0;
    }
    __syncwarp();
    pair_barrier(pair);
    const bool both_ok = xc.m[0].ok && xc.m[1].ok;
    if (!both_ok) {
        if (role == 0 && lane == 0) {
            atomicAdd(&hdr->overflowed, 1ull);
            solve_chain_global_lane0(p, k, start, n, spill, rec_g + k * (long long)max_len, crecp);
        }
        __syncwarp();
        pair_barrier(pair);  // keeps the two warps' barrier counts equal
        return;
    }
    if (role == 0) {
        const float xs = pair_root(xc, 1.f, c_s, lane);
        if (lane == 0) xc.xs = xs;
        __syncwarp();
    }
    pair_barrier(pair);
    const float xs = xc.xs;
    if (role == 0) {
        if (lane == 0) {
            float cc = 0.f;
            if constexpr (P::CREC) cc = c_s;
            p.emit(k, start, s, xs, cc);
        }
        // nodes s-1 .. 0, 32 at a time from the top, composing clips
        float x_next = xs;
        for (int blk = (s - 1) / WARP; blk >= 0; --blk) {
            const int base = blk * WARP;
            const int i = base + lane;
            float lo = -INFINITY, hi = INFINITY;
            if (i < s) {
                const float2 r = recp[i];
                lo = r.x;
                hi = r.y;
            }
            const float xv = clip_suffix(lo, hi, x_next, lane, min(WARP, s - base));
            float cc = 0.f;
            if constexpr (P::CREC) {
                if (i < s) cc = crecp[i];
            }
            if (i < s) p.emit(k, start, i, xv, cc);
            x_next = __shfl_sync(FULL, xv, 0);
        }
    } else {
        // nodes s+1 .. n-1, 32 at a time from the bottom, composing clips
        float x_prev = xs;
        const int m = n - 1 - s;
        for (int blk = 0; blk * WARP < m; ++blk) {
            const int i = s + 1 + blk * WARP + lane;
            float lo = -INFINITY, hi = INFINITY;
            if (i < n) {
                const float2 r = recp[i];
                lo = r.x;
                hi = r.y;
            }
            const float xv = clip_prefix(lo, hi, x_prev, lane, min(WARP, m - blk * WARP));
            float cc = 0.f;
            if constexpr (P::CREC) {
                if (i < n) cc = crecp[i];
            }
            if (i < n) p.emit(k, start, i, xv, cc);
            x_prev = __shfl_sync(FULL, xv, WARP - 1);
        }
    }
}

// ------------------------------------------------------------------------------
// The same middle-rooted split in ONE warp: lanes 0-15 run the left half, lanes
// 16-31 the reversed right half, each half a 16-lane copy of the update above
// (breakpoint k of a half in its lane k, at most 16). Both halves advance in the
// same instructions, so a chain costs half the instructions of the two-warp form;
// a message of more than 16 breakpoints sends the chain to the overflow path.
constexpr int SEG = 16;

// Composition over a 16-lane segment: segment lane j gets the clips of lanes j..15
// applied to x_next (lanes that are not in the block are the identity).
__device__ __forceinline__ float clip_suffix16(float lo, float hi, float x_next, int sl, bool inb)
{
    if (!inb) {
        lo = -INFINITY;
        hi = INFINITY;
    }
#pragma unroll
    for (int o = 1; o < SEG; o <<= 1) {
        const float lo2 = __shfl_down_sync(FULL, lo, o, SEG);
        const float hi2 = __shfl_down_sync(FULL, hi, o, SEG);
        if (sl + o < SEG) {
            const float nlo = clip_to(lo2, lo, hi);
            const float nhi = clip_to(hi2, lo, hi);
            lo = nlo;
            hi = nhi;
        }
    }
    return clip_to(x_next, lo, hi);
}

// Ring form of coop_update for a 16-lane half (TV-l2): the message's breakpoints sit at
// ring positions 0 .. size-1 counted from a head lane, and each lane carries its own
// position `idx`. Removing breakpoints at either end and adding lambda^-, lambda^+ moves
// no data: lambda^- lies on the piece right of the last breakpoint removed on the left,
// so that lane turns into it (with none removed, the lane before the head takes the
// closed-form crossing on the flat left end); the lane after the last kept breakpoint
// turns into lambda^+, the crossing on its predecessor's piece, which every lane passes
// to its successor by one fixed-offset shuffle; and the positions shift by ell - 1. The
// numbers of breakpoints removed on the left and kept through the right are population
// counts of one vote each (m^_i increases along the ring). The lanes that turn into
// lambda^- and lambda^+ store the step's record. The crossings are Sec. 4.1's formula,
// lambda_k + (+-w - v_k) / S_k, kept from falling below lambda_k; the bound at the next
// breakpoint is not applied, since the crossing that is used lies before it
// (v_{k+1} is beyond +-w). What is gone against coop_update are the shuffles that
// shifted the state by a vote-dependent offset. (Computing the predecessor's crossing in
// the successor lane from its shuffled state, to take that one shuffle off the path, was
// slower: the three extra shuffles per step cost more than the latency they hide.)
template <bool ALWAYS>
__device__ __forceinline__ void coop_ring_update(float &lam, float &V, float &T, int &idx,
                                                 int &size, float &w_prev, float ci, float wi,
                                                 int sl, unsigned seg_mask, bool active,
                                                 bool &ovf, float2 *rec)
{
    const bool valid = idx < size;
    const float S = T + 1.f;
    const float v = lam + V - ci;
    // crossings of this lane's piece with -w and +w (not below its breakpoint; the one
    // that is used lies on the piece, before the next breakpoint, as v increases)
    const float rS = __fdividef(1.f, S);
    const float candL = fmaxf(fmaf(-wi - v, rS, lam), lam);
    const float candR = fmaxf(fmaf(wi - v, rS, lam), lam);
    const float candR_prev = __shfl_sync(FULL, candR, (sl - 1) & (SEG - 1), SEG);
    const int ell = __popc(__ballot_sync(FULL, valid && v < -wi) & seg_mask);
    const int nle = __popc(__ballot_sync(FULL, valid && v <= wi) & seg_mask);
    // lambda^+ takes ring position max(nle, ell) (one past the last kept breakpoint), and
    // the new message holds the kept ones between lambda^- and lambda^+
    const int hpos = max(nle, ell);
    const int nsize = hpos - ell + 2;
    ovf = ovf || ((ALWAYS || active) && nsize > SEG);
    if (ALWAYS || active) {
        const int lpos = ell - 1;
        const bool is_lm = idx == (lpos & (SEG - 1));
        const bool is_hp = idx == (hpos & (SEG - 1));
        const float lm = ell == 0 ? ci - wi + w_prev : candL;
        const float hp = hpos == 0 ? ci + wi + w_prev : candR_prev;
        if (is_lm) rec->x = lm;
        if (is_hp) rec->y = hp;
        lam = is_lm ? lm : (is_hp ? hp : lam);
        V = is_lm ? -wi : (is_hp ? wi : v);
        T = is_lm ? (ell == 0 ? 1.f : S) : (is_hp ? 0.f : S);
        idx = (idx - lpos) & (SEG - 1);
        size = nsize;
        w_prev = wi;
    }
}

// clip_suffix16's composition for two segments at once (their rounds interleaved, since
// neither waits for x_next): lane j of each gets the clips of lanes j..15 composed.
__device__ __forceinline__ void clip_compose16_pair(float &lo0, float &hi0, bool inb0, float &lo1,
                                                    float &hi1, bool inb1, int sl)
{
    if (!inb0) {
        lo0 = -INFINITY;
        hi0 = INFINITY;
    }
    if (!inb1) {
        lo1 = -INFINITY;
        hi1 = INFINITY;
    }
#pragma unroll
    for (int o = 1; o < SEG; o <<= 1) {
        const float a = __shfl_down_sync(FULL, lo0, o, SEG);
        const float b = __shfl_down_sync(FULL, hi0, o, SEG);
        const float c = __shfl_down_sync(FULL, lo1, o, SEG);
        const float d = __shfl_down_sync(FULL, hi1, o, SEG);
        if (sl + o < SEG) {
            const float nlo0 = clip_to(a, lo0, hi0), nhi0 = clip_to(b, lo0, hi0);
            const float nlo1 = clip_to(c, lo1, hi1), nhi1 = clip_to(d, lo1, hi1);
            lo0 = nlo0;
            hi0 = nhi0;
            lo1 = nlo1;
            hi1 = nhi1;
        }
    }
}

// coop_ring_update for the general unary a_i z^2 / 2 - b_i z and slopes [w^-_i, w^+_i]
// (coop_update_g's arithmetic in the ring form; wl_prev is w^-_{i-1}).
template <bool ALWAYS>
__device__ __forceinline__ void coop_ring_update_g(float &lam, float &V, float &T, int &idx,
                                                   int &size, float &wl_prev, float ai, float bi,
                                                   float wl, float wh, int sl, unsigned seg_mask,
                                                   bool active, bool &ovf, float2 *rec)
{
    const bool valid = idx < size;
    const float S = T + ai;
    const float v = fmaf(ai, lam, V) - bi;
    const float rS = __fdividef(1.f, S);
    const float candL = fmaxf(fmaf(wl - v, rS, lam), lam);
    const float candR = fmaxf(fmaf(wh - v, rS, lam), lam);
    const float candR_prev = __shfl_sync(FULL, candR, (sl - 1) & (SEG - 1), SEG);
    const int ell = __popc(__ballot_sync(FULL, valid && v < wl) & seg_mask);
    const int nle = __popc(__ballot_sync(FULL, valid && v <= wh) & seg_mask);
    const int hpos = max(nle, ell);
    const int nsize = hpos - ell + 2;
    ovf = ovf || ((ALWAYS || active) && nsize > SEG);
    if (ALWAYS || active) {
        const int lpos = ell - 1;
        const bool is_lm = idx == (lpos & (SEG - 1));
        const bool is_hp = idx == (hpos & (SEG - 1));
        // on the flat left end m^_i = w^-_{i-1} + a_i z - b_i
        const float lm = ell == 0 ? (bi + wl - wl_prev) / ai : candL;
        const float hp = hpos == 0 ? (bi + wh - wl_prev) / ai : candR_prev;
        if (is_lm) rec->x = lm;
        if (is_hp) rec->y = hp;
        lam = is_lm ? lm : (is_hp ? hp : lam);
        V = is_lm ? wl : (is_hp ? wh : v);
        T = is_lm ? (ell == 0 ? ai : S) : (is_hp ? 0.f : S);
        idx = (idx - lpos) & (SEG - 1);
        size = nsize;
        wl_prev = wl;
    }
}

// Policies whose edge weights are one value for the whole chain (a scaled lambda) say
// so with `static constexpr bool UNIFORM_W = true`: the halves then take each step's
// weight from their own lane instead of a shuffle.
template <class P, class = void>
struct coop_uniform_w : std::false_type {};
template <class P>
struct coop_uniform_w<P, std::enable_if_t<P::UNIFORM_W>> : std::true_type {};

// 16 update steps of both halves (positions base..base+15). FB: every step of the block
// is an update in both halves (no root step, no tail). UW: one weight for the chain.
template <bool FB, bool UW, class P>
__device__ __forceinline__ void coop_halves_block(
    const P &p, typename P::Acc &acc, long long k, long long start, int n, int base, int cntw,
    int half, int sl, int seg_shift, float cv, float wv, float wsel,
    const typename P::Raw &raw_next, float2 *rec_b, float &lam, float &V, float &T, int &idx,
    int &size, float &w_prev, float &c_s, bool &ovf)
{
    // the block's c_i (and w_i) broadcast up front, off the steps' critical path
    float cis[SEG], wis[SEG];
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
        cis[j] = __shfl_sync(FULL, cv, j, SEG);
        if constexpr (!UW) wis[j] = __shfl_sync(FULL, wsel, j, SEG);
    }
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
        const int qq = base + j;
        const float ci = cis[j];
        float wi = wv;
        if constexpr (!UW) {
            wi = wis[j];
            if (j == SEG - 1) {
                // the right half's last step takes the weight staged with the next block
                float c2, w2;
                const int qn = base + SEG;
                p.unary(k, start, n, qn < cntw ? (half == 0 ? qn : n - 1 - qn) : n, raw_next, c2,
                        w2, acc);
                const float w_nb = __shfl_sync(FULL, w2, 0, SEG);
                if (half == 1) wi = w_nb;
            }
        }
        const bool stepping = FB || qq < cntw - 1;
        if constexpr (!FB) {
            if (half == 0 && qq == cntw - 1) c_s = ci;
        }
        coop_ring_update<FB>(lam, V, T, idx, size, w_prev, ci, wi, sl, 0xFFFFu << seg_shift,
                             stepping, ovf, rec_b + j);
    }
}

template <class P>
__device__ void coop_solve_chain_halves(const P &p, typename P::Acc &acc, long long k,
                                        long long start, int n, int lane, PairXchg &xc,
                                        float2 *sm_rec, float *sm_crec, int smem_nodes,
                                        float2 *rec_g, float *crec_g, float2 *spill,
                                        WsHeader *hdr)
{
    const int max_len = p.max_len();
    const bool in_smem = n <= smem_nodes;
    float2 *recp = in_smem ? sm_rec : rec_g + k * (long long)max_len;
    float *crecp = nullptr;
    if constexpr (P::CREC) crecp = in_smem ? sm_crec : crec_g + k * (long long)max_len;
    const int s = n / 2;
    const int half = lane >> 4, sl = lane & (SEG - 1), seg_shift = half * SEG;
    // the left half walks nodes 0..s, the right half n-1..s (node s for its weight)
    const int cntw = half == 0 ? s + 1 : n - s;
    const int cnt_all = (s + 1 > n - s) ? s + 1 : n - s;
    auto node = [&](int q) { return half == 0 ? q : n - 1 - q; };
    auto fetch_at = [&](int q, typename P::Raw &r) {
        p.fetch(k, start, n, q < cntw ? node(q) : n, r);
    };

    // Message state of this half; the empty message (size 0, w_prev = 0) makes
    // the first update produce m_{0,1} = clip(z - c_0, -w_0, w_0) exactly.
    float lam = 0.f, V = 0.f, T = 0.f, w_prev = 0.f, c_s = 0.f;
    int size = 0, idx = sl;  // the message in ring order; idx: this lane's ring position
    bool ok = true, ovf = false;
    typename P::Raw raw, raw_next{};
    fetch_at(sl, raw);
    constexpr bool UW = coop_uniform_w<P>::value;
    const int cnt_lo = (s + 1 < n - s) ? s + 1 : n - s;  // the shorter half's positions
    const int nblocks = (cnt_all + SEG - 1) / SEG;
    for (int blk = 0; blk < nblocks; ++blk) {
        const int base = blk * SEG;
        if (blk + 1 < nblocks) fetch_at(base + SEG + sl, raw_next);
        const int q = base + sl;
        const int i_l = q < cntw ? node(q) : n;
        float cv, wv;
        p.unary(k, start, n, i_l, raw, cv, wv, acc);
        if constexpr (P::CREC) {
            if (q < cntw && (half == 0 || i_l != s)) crecp[i_l] = cv;  // node s: left half
        }
        // the right half steps node i with the weight of edge (i-1, i): that of the
        // next position (the next lane; for the segment's last lane, the first
        // position of the next block, read when the last step needs it)
        float wsel = wv;
        if constexpr (!UW) {
            const float wr = __shfl_down_sync(FULL, wv, 1, SEG);
            wsel = half == 0 ? wv : wr;
        }
        // records of this block's steps at slots base + j: the left half's are its nodes,
        // the right half's are mirrored (node i at slot n + s - i, from s + 1 up), so that
        // both halves store forwards from one pointer
        float2 *rec_b = recp + (half == 0 ? base : s + 1 + base);
        if (ok) {
            if (base + SEG < cnt_lo)
                coop_halves_block<true, UW>(p, acc, k, start, n, base, cntw, half, sl, seg_shift,
                                            cv, wv, wsel, raw_next, rec_b, lam, V, T, idx, size,
                                            w_prev, c_s, ovf);
            else
                coop_halves_block<false, UW>(p, acc, k, start, n, base, cntw, half, sl, seg_shift,
                                             cv, wv, wsel, raw_next, rec_b, lam, V, T, idx, size,
                                             w_prev, c_s, ovf);
            ok = !__any_sync(FULL, ovf);
        }
        raw = raw_next;
    }
    __syncwarp();
    if (!ok) {
        // a half outgrew 16 breakpoints: solve the chain from one end with all 32 lanes
        // (which itself falls back to lane 0 beyond 32)
        coop_solve_chain(p, acc, k, start, n, lane, sm_rec, sm_crec, smem_nodes, rec_g, crec_g,
                         spill, hdr);
        return;
    }
    PairMsg &mine = xc.m[half];
    if (idx < size) {  // back to ascending order from entry 0
        mine.lam[idx] = lam;
        mine.val[idx] = V;
    }
    if (sl == 0) mine.size = size;
    __syncwarp();
    const float cs_all = __shfl_sync(FULL, c_s, 0);
    const float xs = pair_root(xc, 1.f, cs_all, lane);
    if (lane == 0) {
        float cc = 0.f;
        if constexpr (P::CREC) cc = cs_all;
        p.emit(k, start, s, xs, cc);
    }
    // backward, 16 nodes per half and step, outward from s: the left half takes
    // nodes top-down (lane j: node blk*16 + j), the right half bottom-up with its
    // lanes reversed (lane j: node s+1 + t*16 + 15 - j), so that both compose their
    // clips as a suffix over the segment
    const int nbl_l = (s + SEG - 1) / SEG;
    const int nbl_r = (n - 1 - s + SEG - 1) / SEG;
    const int nbb = nbl_l > nbl_r ? nbl_l : nbl_r;
    auto seg_node = [&](int t, int &i, bool &inb) {
        if (half == 0) {
            const int blk = nbl_l - 1 - t;
            i = blk * SEG + sl;
            inb = blk >= 0 && i < s;
        } else {
            i = s + 1 + t * SEG + (SEG - 1 - sl);
            inb = t < nbl_r && i < n;
        }
    };
    auto load_rec = [&](int i, bool inb, float &lo, float &hi) {
        lo = -INFINITY;
        hi = INFINITY;
        if (inb) {
            const float2 r = recp[half == 0 ? i : n + s - i];  // right half: mirrored slots
            lo = r.x;
            hi = r.y;
        }
    };
    auto finish = [&](int i, bool inb, float xv) {
        if (inb) {
            float cc = 0.f;
            if constexpr (P::CREC) cc = crecp[i];
            p.emit(k, start, i, xv, cc);
        }
    };
    // two segments per round: their compositions do not wait for x_next, only the final
    // clips do
    float x_next = xs;
    for (int t = 0; t < nbb; t += 2) {
        int i0, i1;
        bool in0, in1;
        seg_node(t, i0, in0);
        seg_node(t + 1, i1, in1);
        if (t + 1 >= nbb) in1 = false;
        float lo0, hi0, lo1, hi1;
        load_rec(i0, in0, lo0, hi0);
        load_rec(i1, in1, lo1, hi1);
        clip_compose16_pair(lo0, hi0, in0, lo1, hi1, in1, sl);
        const float x0 = clip_to(x_next, lo0, hi0);
        finish(i0, in0, x0);
        x_next = __shfl_sync(FULL, x0, 0, SEG);
        const float x1 = clip_to(x_next, lo1, hi1);
        finish(i1, in1, x1);
        x_next = __shfl_sync(FULL, x1, 0, SEG);
    }
}

// ------------------------------------------------------------------------------
// General convex chains (Sec. 4, Sec. 4.1): policies with unary_g give, per node,
// a_i > 0, b_i and the pairwise slopes [w^-_i, w^+_i] of edge (i, i+1).
template <class P, class = void>
struct has_unary_g : std::false_type {};
template <class P>
struct has_unary_g<P, std::void_t<decltype(&P::unary_g)>> : std::true_type {};

// Overflow path of the general chain: lane 0, the two-ended array of Sec. 4.1 (2n+2
// entries (lambda, s), true slope s + abar_i, abar_i = sum a_k) in global memory.
template <class P>
__device__ void solve_chain_general_lane0(const P &p, long long k, long long start, int n,
                                          float2 *D, float2 *rec)
{
    float a, b, wl, wh;
    p.unary_g_direct(0, n, k, start, a, b, wl, wh);
    if (n == 1) {
        p.emit(k, start, 0, b / a, 0.f);
        return;
    }
    float abar = a;
    int front = n, back = n + 1;
    D[front] = make_float2((b + wl) / a, 0.f);
    D[back] = make_float2((b + wh) / a, -abar);
    rec[0] = make_float2(D[front].x, D[back].x);
    float wl_prev = wl, wh_prev = wh, xlast = 0.f;
    for (int i = 1; i < n; ++i) {
        p.unary_g_direct(i, n, k, start, a, b, wl, wh);
        abar += a;
        int pp = front;
        float v = fmaf(a, D[pp].x, wl_prev) - b;
        int last_popped;
        float lm, lm_s;
        if (v >= wl) {
            last_popped = front - 1;
            lm = D[pp].x + (wl - v) / a;
            lm_s = a - abar;
        } else {
            while (pp < back) {
                const float vq = v + (D[pp].y + abar) * (D[pp + 1].x - D[pp].x);
                if (!(vq < wl)) break;
                ++pp;
                v = vq;
            }
            last_popped = pp;
            lm = D[pp].x + (wl - v) / (D[pp].y + abar);
            lm_s = D[pp].y;
        }
        float hp;
        int new_back_last;
        if (back > last_popped) {
            int q = back;
            float vr = fmaf(a, D[q].x, wh_prev) - b;
            if (vr <= wh) {
                hp = D[q].x + (wh - vr) / a;
                new_back_last = back;
            } else {
                for (;;) {
                    if (q - 1 > last_popped) {
                        const float slope = D[q - 1].y + abar;
                        const float vprev = vr - slope * (D[q].x - D[q - 1].x);
                        if (vprev > wh) {
                            --q;
                            vr = vprev;
                            continue;
                        }
                        hp = D[q].x - (vr - wh) / slope;
                    } else {
                        hp = D[q].x - (vr - wh) / (lm_s + abar);
                    }
                    break;
                }
                new_back_last = q - 1;
            }
        } else {
            hp = lm + (wh - wl) / (lm_s + abar);
            new_back_last = last_popped;
        }
        front = last_popped;
        D[front] = make_float2(lm, lm_s);
        back = (new_back_last > front ? new_back_last : front) + 1;
        D[back] = make_float2(hp, -abar);
        if (i == n - 1) xlast = 0.5f * (lm + hp);
        else rec[i] = make_float2(lm, hp);
        wl_prev = wl;
        wh_prev = wh;
    }
    float xv = xlast;
    p.emit(k, start, n - 1, xv, 0.f);
    for (int i = n - 2; i >= 0; --i) {
        const float2 r = rec[i];
        xv = clip_to(xv, r.x, r.y);
        p.emit(k, start, i, xv, 0.f);
    }
}

// One general chain by one warp from one end (any length).
template <class P>
__device__ void coop_solve_chain_general(const P &p, typename P::Acc &acc, long long k,
                                         long long start, int n, int lane, float2 *sm_rec,
                                         int smem_nodes, float2 *rec_g, float2 *spill,
                                         WsHeader *hdr)
{
    const int max_len = p.max_len();
    float2 *recp = n <= smem_nodes ? sm_rec : rec_g + k * (long long)max_len;
    // empty message: the first update produces m_{0,1} = clip(a_0 z - b_0, w^-_0, w^+_0)
    float lam = 0.f, V = 0.f, T = 0.f, wl_prev = 0.f, xlast = 0.f;
    int size = 0;
    bool ok = true, ovf = false;
    typename P::Raw raw, raw_next{};
    p.fetch(k, start, n, lane, raw);
    const int nblocks = (n + WARP - 1) / WARP;
    for (int blk = 0; blk < nblocks; ++blk) {
        const int base = blk * WARP;
        if (blk + 1 < nblocks) p.fetch(k, start, n, base + WARP + lane, raw_next);
        float av, bv, wlv, whv;
        p.unary_g(k, start, n, base + lane, raw, av, bv, wlv, whv, acc);
        const int cnt = min(WARP, n - base);
        if (ok) {
            for (int j = 0; j < cnt; ++j) {
                const int i = base + j;
                const float ai = __shfl_sync(FULL, av, j), bi = __shfl_sync(FULL, bv, j);
                const float wl = (i < n - 1) ? __shfl_sync(FULL, wlv, j) : 0.f;
                const float wh = (i < n - 1) ? __shfl_sync(FULL, whv, j) : 0.f;
                float lmv, hpv;
                coop_update_g<WARP>(lam, V, T, size, wl_prev, ai, bi, wl, wh, lane, 0, true,
                                    ovf, lmv, hpv);
                if (i == n - 1) xlast = (n == 1) ? bi / ai : 0.5f * (lmv + hpv);
                else if (lane == 0) recp[i] = make_float2(lmv, hpv);
            }
            ok = !ovf;
        }
        raw = raw_next;
    }
    __syncwarp();
    if (!ok) {
        if (lane == 0) {
            atomicAdd(&hdr->overflowed, 1ull);
            solve_chain_general_lane0(p, k, start, n, spill, rec_g + k * (long long)max_len);
        }
        __syncwarp();
        return;
    }
    float x_next = xlast;
    for (int blk = nblocks - 1; blk >= 0; --blk) {
        const int i = blk * WARP + lane;
        float lo = -INFINITY, hi = INFINITY;
        if (i < n - 1) {
            const float2 r = recp[i];
            lo = r.x;
            hi = r.y;
        }
        const float xv = clip_suffix(lo, hi, x_next, lane, min(WARP, n - blk * WARP));
        if (i < n) p.emit(k, start, i, xv, 0.f);
        x_next = __shfl_sync(FULL, xv, 0);
    }
}

// One general chain of kSplitMinLen nodes or more: rooted at its middle node, the two
// forward passes in the warp's two 16-lane halves (as coop_solve_chain_halves). The
// reversed right half sees edge (i-1, i) with the slopes [-w^+_{i-1}, -w^-_{i-1}].
template <class P>
__device__ void coop_solve_chain_halves_general(const P &p, typename P::Acc &acc, long long k,
                                                long long start, int n, int lane, PairXchg &xc,
                                                float2 *sm_rec, int smem_nodes, float2 *rec_g,
                                                float2 *spill, WsHeader *hdr)
{
    const int max_len = p.max_len();
    float2 *recp = n <= smem_nodes ? sm_rec : rec_g + k * (long long)max_len;
    const int s = n / 2;
    const int half = lane >> 4, sl = lane & (SEG - 1), seg_shift = half * SEG;
    const int cntw = half == 0 ? s + 1 : n - s;
    const int cnt_all = (s + 1 > n - s) ? s + 1 : n - s;
    auto node = [&](int q) { return half == 0 ? q : n - 1 - q; };
    auto fetch_at = [&](int q, typename P::Raw &r) {
        p.fetch(k, start, n, q < cntw ? node(q) : n, r);
    };
    float lam = 0.f, V = 0.f, T = 0.f, wl_prev = 0.f, a_s = 1.f, b_s = 0.f;
    int size = 0, idx = sl;  // the message in ring order; idx: this lane's ring position
    bool ok = true, ovf = false;
    typename P::Raw raw, raw_next{};
    fetch_at(sl, raw);
    const int nblocks = (cnt_all + SEG - 1) / SEG;
    for (int blk = 0; blk < nblocks; ++blk) {
        const int base = blk * SEG;
        if (blk + 1 < nblocks) fetch_at(base + SEG + sl, raw_next);
        const int q = base + sl;
        const int i_l = q < cntw ? node(q) : n;
        float av, bv, wlv, whv;
        p.unary_g(k, start, n, i_l, raw, av, bv, wlv, whv, acc);
        // right half: the next position's edge, reversed
        const float wlr = __shfl_down_sync(FULL, wlv, 1, SEG);
        const float whr = __shfl_down_sync(FULL, whv, 1, SEG);
        const float wl_sel = half == 0 ? wlv : -whr;
        const float wh_sel = half == 0 ? whv : -wlr;
        if (ok) {
#pragma unroll
            for (int j = 0; j < SEG; ++j) {
                const int qq = base + j;
                const float ai = __shfl_sync(FULL, av, j, SEG);
                const float bi = __shfl_sync(FULL, bv, j, SEG);
                float wl = __shfl_sync(FULL, wl_sel, j, SEG);
                float wh = __shfl_sync(FULL, wh_sel, j, SEG);
                if (j == SEG - 1) {
                    float a2, b2, wl2, wh2;
                    p.unary_g(k, start, n, base + SEG < cntw ? node(base + SEG) : n, raw_next, a2,
                              b2, wl2, wh2, acc);
                    const float nl = __shfl_sync(FULL, wl2, 0, SEG);
                    const float nh = __shfl_sync(FULL, wh2, 0, SEG);
                    if (half == 1) {
                        wl = -nh;
                        wh = -nl;
                    }
                }
                const bool stepping = qq < cntw - 1;
                if (half == 0 && qq == cntw - 1) {
                    a_s = ai;
                    b_s = bi;
                }
                coop_ring_update_g<false>(lam, V, T, idx, size, wl_prev, ai, bi, wl, wh, sl,
                                          0xFFFFu << seg_shift, stepping, ovf, recp + node(qq));
            }
            ok = !__any_sync(FULL, ovf);
        }
        raw = raw_next;
    }
    __syncwarp();
    if (!ok) {
        // a half outgrew 16 breakpoints: the whole warp from one end (then lane 0)
        coop_solve_chain_general(p, acc, k, start, n, lane, sm_rec, smem_nodes, rec_g, spill, hdr);
        return;
    }
    PairMsg &mine = xc.m[half];
    if (idx < size) {  // back to ascending order from entry 0
        mine.lam[idx] = lam;
        mine.val[idx] = V;
    }
    if (sl == 0) mine.size = size;
    __syncwarp();
    const float as_all = __shfl_sync(FULL, a_s, 0), bs_all = __shfl_sync(FULL, b_s, 0);
    const float xs = pair_root(xc, as_all, bs_all, lane);
    if (lane == 0) p.emit(k, start, s, xs, 0.f);
    const int nbl_l = (s + SEG - 1) / SEG;
    const int nbl_r = (n - 1 - s + SEG - 1) / SEG;
    const int nbb = nbl_l > nbl_r ? nbl_l : nbl_r;
    float x_next = xs;
    for (int t = 0; t < nbb; ++t) {
        int i;
        bool inb;
        if (half == 0) {
            const int blk = nbl_l - 1 - t;
            i = blk * SEG + sl;
            inb = blk >= 0 && i < s;
        } else {
            i = s + 1 + t * SEG + (SEG - 1 - sl);
            inb = t < nbl_r && i < n;
        }
        float lo = -INFINITY, hi = INFINITY;
        if (inb) {
            const float2 r = recp[i];
            lo = r.x;
            hi = r.y;
        }
        const float xv = clip_suffix16(lo, hi, x_next, sl, inb);
        if (inb) p.emit(k, start, i, xv, 0.f);
        x_next = __shfl_sync(FULL, xv, 0, SEG);
    }
}

// Two warps per chain: warp pair q of a block solves chain blockIdx.x * pairs + q.
// Shared memory: one PairXchg per pair, then the pairs' records (and c records).
template <class P>
__global__ void __launch_bounds__(256) coop_pair_kernel(P p_in, float2 *rec_g, float *crec_g,
                                                        float2 *spill, WsHeader *hdr,
                                                        int smem_nodes)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    P p = p_in;
    if (!p.resolve()) return;
    const int lane = threadIdx.x & (WARP - 1);
    const int warp = threadIdx.x / WARP;
    const int pairs = blockDim.x / (2 * WARP);
    const int pair = warp >> 1, role = warp & 1;
    PairXchg *xch = reinterpret_cast<PairXchg *>(smem_raw);
    float2 *sm_rec = reinterpret_cast<float2 *>(xch + pairs) + (size_t)pair * smem_nodes;
    float *sm_crec = reinterpret_cast<float *>(reinterpret_cast<float2 *>(xch + pairs) +
                                               (size_t)pairs * smem_nodes) +
                     (size_t)pair * smem_nodes;
    const long long k = (long long)blockIdx.x * pairs + pair;  // this pair's chain
    typename P::Acc acc;
    p.acc_init(acc);
    long long start = 0;
    int n = 0;
    if (k < p.num_chains()) {
        if (!p.chain(k, start, n)) {
            if (lane == 0 && role == 0) atomicOr(&hdr->status, ERR_BAD_CHAIN);
            n = 0;
        }
    }
    if (n == 0 || (n < kSplitMinLen && role == 1)) {
        p.finish_empty();
        return;
    }
    if (n < kSplitMinLen) {
        coop_solve_chain(p, acc, k, start, n, lane, sm_rec, sm_crec, smem_nodes, rec_g,
                         crec_g, spill + p.spill_off(k, start), hdr);
    } else {
        coop_solve_chain_split(p, acc, k, start, n, lane, role, pair, xch[pair], sm_rec,
                               sm_crec, smem_nodes, rec_g, crec_g,
                               spill + p.spill_off(k, start), hdr);
    }
    p.finish(acc, lane);
}

// One warp per chain; with HALVES, chains of kSplitMinLen nodes or more are rooted
// at their middle node and solved as two 16-lane halves. Shared memory: (HALVES)
// one PairXchg per warp, then the warps' records (and c records). Launched with at
// most 256 threads; no launch bound, which on this target would cap the update at 64
// registers and spill it.
template <class P, bool HALVES>
__global__ void coop_chain_kernel(P p_in, float2 *rec_g, float *crec_g,
                                                         float2 *spill, WsHeader *hdr,
                                                         int smem_nodes)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    P p = p_in;
    if (!p.resolve()) return;
    const int lane = threadIdx.x & (WARP - 1);
    const int warp = threadIdx.x / WARP;
    const int wpb = blockDim.x / WARP;
    PairXchg *xch = reinterpret_cast<PairXchg *>(smem_raw);
    unsigned char *rec_base = smem_raw + (HALVES ? wpb * sizeof(PairXchg) : 0);
    float2 *sm_rec = reinterpret_cast<float2 *>(rec_base) + (size_t)warp * smem_nodes;
    float *sm_crec = reinterpret_cast<float *>(reinterpret_cast<float2 *>(rec_base) +
                                               (size_t)wpb * smem_nodes) +
                     (size_t)warp * smem_nodes;
    const long long k = (long long)blockIdx.x * wpb + warp;  // this warp's chain
    typename P::Acc acc;
    p.acc_init(acc);
    long long start = 0;
    int n = 0;
    if (k < p.num_chains()) {
        if (!p.chain(k, start, n)) {
            if (lane == 0) atomicOr(&hdr->status, ERR_BAD_CHAIN);
            n = 0;
        }
    }
    if (n == 0) {
        p.finish_empty();
        return;
    }
    if constexpr (has_unary_g<P>::value) {
        if (HALVES && n >= kSplitMinLen)
            coop_solve_chain_halves_general(p, acc, k, start, n, lane, xch[warp], sm_rec,
                                            smem_nodes, rec_g, spill + p.spill_off(k, start), hdr);
        else
            coop_solve_chain_general(p, acc, k, start, n, lane, sm_rec, smem_nodes, rec_g,
                                     spill + p.spill_off(k, start), hdr);
    } else {
        if (HALVES && n >= kSplitMinLen)
            coop_solve_chain_halves(p, acc, k, start, n, lane, xch[warp], sm_rec, sm_crec,
                                    smem_nodes, rec_g, crec_g, spill + p.spill_off(k, start), hdr);
        else
            coop_solve_chain(p, acc, k, start, n, lane, sm_rec, sm_crec, smem_nodes, rec_g, crec_g,
                             spill + p.spill_off(k, start), hdr);
    }
    p.finish(acc, lane);
}

}  // namespace tvk
