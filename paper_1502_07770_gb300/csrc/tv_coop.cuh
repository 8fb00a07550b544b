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

// The warp-cooperative message update of one node (abar = i + 1 is implicit).
// Lane k holds breakpoint lambda_k of the message m_{i-1,i} and its value V_k
// there (valid for k < size); lam0/lamL are the first and last breakpoint, whose
// values are -w_{i-1} and +w_{i-1}. Storing values instead of the implicit slopes
// of Sec. 4.1 makes transformation (a), m^_i = m_{i-1,i} + z - c_i, the lane-local
// update v_k = V_k + lambda_k - c_i (no scan), and each new breakpoint is where
// the linear piece of m^_i between two neighbouring breakpoints crosses -w_i or
// +w_i. The message is the same piecewise-linear function; the values are also
// more precise in FP32, since they are never rebuilt through large slopes.
// Returns false (state untouched) if the new message would exceed 32 breakpoints.
__device__ __forceinline__ float seg_frac(float num, float den)
{
    // fraction along a segment, clamped to [0, 1] (0 for a zero-length segment)
    return fminf(fmaxf(__fdividef(num, den), 0.f), 1.f);
}

__device__ __forceinline__ bool coop_step(float &lam, float &V, int &size, float &lam0,
                                          float &lamL, float &w_prev, float ci, float wi,
                                          int lane, float &lm, float &hp)
{
    const bool valid = lane < size;
    const bool last = lane == size - 1;
    const float v = V + lam - ci;           // m^_i at breakpoint `lane`
    const float v0 = lam0 - ci - w_prev;    // m^_i at the first breakpoint
    float lam_n = __shfl_down_sync(FULL, lam, 1);
    float v_n = __shfl_down_sync(FULL, v, 1);
    // left scan: breakpoints with m^_i < -w_i (a prefix); right scan: those with
    // m^_i > w_i among the rest (a suffix). The breakpoints removed on the left have
    // m^_i < -w_i <= w_i, so the last one not above w_i is never left of ell - 1.
    const int ell = min((int)__reduce_min_sync(FULL, (unsigned)((valid && v >= -wi) ? lane : WARP)),
                        size);                                          // removed on the left
    const int kl = __reduce_max_sync(FULL, (valid && v <= wi) ? lane : -1);
    const int keep_last = kl > ell - 1 ? kl : ell - 1;  // last kept breakpoint (-1: none)
    const int K = keep_last - ell + 1;
    if (K + 2 > WARP) return false;

    // Crossings of -w_i and +w_i on the piece right of this breakpoint: between it
    // and the next one (clamped to the segment), or, for the last breakpoint, on the
    // right end piece of slope a_i = 1.
    float fl, fr;
    if (last) {
        fl = -wi - v;
        fr = wi - v;
        lam_n = lam + 1.f;
    } else {
        const float dv = v_n - v;
        fl = seg_frac(-wi - v, dv);
        fr = seg_frac(wi - v, dv);
    }
    const float dl = lam_n - lam;
    const float candL = fmaf(fl, dl, lam);
    const float candR = fmaf(fr, dl, lam);
    // lambda^- lies on the piece right of the last breakpoint removed on the left,
    // lambda^+ on the piece right of the last one kept (which may hold both); with
    // none, on the left end piece of slope 1.
    const float gl = __shfl_sync(FULL, candL, (ell - 1) & (WARP - 1));
    const float gr = __shfl_sync(FULL, candR, keep_last & (WARP - 1));
    lm = (ell == 0) ? lam0 - (v0 + wi) : gl;
    hp = (keep_last < 0) ? lam0 + (wi - v0) : gr;
    // new message m_{i,i+1}: lambda^- (value -w_i), kept breakpoints with their
    // values unchanged by the clip, lambda^+ (value +w_i)
    const int src = (lane - 1 + ell) & (WARP - 1);
    const float nl = __shfl_sync(FULL, lam, src);
    const float nv = __shfl_sync(FULL, v, src);
    lam = (lane == 0) ? lm : ((lane == K + 1) ? hp : nl);
    V = (lane == 0) ? -wi : ((lane == K + 1) ? wi : nv);
    size = K + 2;
    lam0 = lm;
    lamL = hp;
    w_prev = wi;
    return true;
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

    float lam = 0.f, s = 0.f /* value at the breakpoint */, lam0 = 0.f, lamL = 0.f, w_prev = 0.f;
    int size = 0;
    bool ok = true;
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
                    lmv = ci - wi;
                    hpv = ci + wi;
                    if (n == 1) {
                        xlast = ci;
                        break;
                    }
                    lam = (lane == 0) ? lmv : hpv;
                    s = (lane == 0) ? -wi : wi;  // values of m_{0,1} at its breakpoints
                    size = 2;
                    lam0 = lmv;
                    lamL = hpv;
                    w_prev = wi;
                } else if (!coop_step(lam, s, size, lam0, lamL, w_prev, ci, wi, lane, lmv,
                                      hpv)) {
                    ok = false;
                    break;
                }
                if (i == n - 1) xlast = 0.5f * (lmv + hpv);
                else if (lane == 0) recp[i] = make_float2(lmv, hpv);
            }
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

template <class P>
__global__ void __launch_bounds__(256) coop_chain_kernel(P p_in, float2 *rec_g, float *crec_g,
                                                         float2 *spill, WsHeader *hdr,
                                                         int smem_nodes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    P p = p_in;
    if (!p.resolve()) return;
    const int lane = threadIdx.x & (WARP - 1);
    const int warp = threadIdx.x / WARP;
    const int wpb = blockDim.x / WARP;
    float2 *sm_rec = reinterpret_cast<float2 *>(smem_raw) + (size_t)warp * smem_nodes;
    float *sm_crec = reinterpret_cast<float *>(reinterpret_cast<float2 *>(smem_raw) +
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
    coop_solve_chain(p, acc, k, start, n, lane, sm_rec, sm_crec, smem_nodes, rec_g, crec_g,
                     spill + p.spill_off(k, start), hdr);
    p.finish(acc, lane);
}

}  // namespace tvk
