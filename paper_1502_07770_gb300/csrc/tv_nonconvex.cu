// Chains with continuous piecewise-linear unaries and truncated TV (Sec. 3):
//     x* in argmin_x sum_i f_i(x_i) + sum_{i<n} min(w_i |x_{i+1} - x_i|, C_i),
// f_i any continuous piecewise-linear function bounded below (a stereo matching cost,
// say), w_i >= 0, C_i >= 0 (C_i = +inf: plain TV). Dynamic programming on the chain
// (eq. Message:update): M^_i = f_i + M_{i-1,i}, M_{i,i+1} = M^_i (x) min(w_i|.|, C_i), the
// min-convolution taken as the three consecutive ones of Prop. ConsecutiveMinConvolution:
// with f^1 (Algorithm 1), with f^2 (Algorithm 1 on the mirrored function) and with f^3
// (min(h, min h + C)).
//
// Two warps per chain, one per half of a chain rooted at its middle node (see
// nc_chain_kernel). A message is a list of breakpoints (lambda_p, h(lambda_p)) in shared
// memory plus the slopes of its two ends; each lane owns a contiguous chunk of the list.
//  - sum: the two sorted lists are merged by merge-path partitioning (one binary search
//    per lane, then a sequential merge of the lane's output chunk), every point taking
//    the other function's value by interpolation;
//  - Algorithm 1 as a scan: with g(z) = h(z) - w z, (h (x) f^1)(z) = w z + min_{y<=z} g(y),
//    so a warp prefix-minimum of g over the breakpoints decides which points stay (those
//    on the running minimum) and where a falling segment re-crosses the running minimum
//    (the new breakpoint of Algorithm 1); survivors are compacted by a warp scan of
//    counts. f^2 is the same pass run from the right end with g(z) = h(z) + w z;
//  - f^3: a warp minimum gives min h; points are clipped to min h + C, crossings added.
// Values are kept relative to the minimum of M^_i (the minimum is the same after every
// min-convolution, since each f^k >= 0 with f^k(0) = 0); the minima are summed in FP64 into
// the chain's optimum energy. Every M^_i goes to the workspace; the backward pass takes
// the root's x in argmin M^_root and, outwards, x_i = pi_i(x_j) (j the neighbour on the
// root side) from the definition of pi as an argmin of M^_i(z) + min(w |x_j - z|, C) over
// z, evaluated at every breakpoint of M^_i and at x_j, x_j - C/w, x_j + C/w (the first
// minimum in that order).
#include <cuda_runtime.h>

#include <algorithm>

#include "tv_launch.cuh"

using namespace tvk;
using namespace tvh;

namespace {

constexpr int kNcMaxWarps = 4;

// warps per block: as many as fit three message buffers each in ~220 KB of shared memory
// (at least the two warps of one chain: 2 * 24 * 4096 bytes fit)
int nc_warps(int T) { return std::max(2, std::min(kNcMaxWarps, (220 * 1024) / (24 * T))); }

struct NcArgs {
    const int64_t *uoff;  // node -> first breakpoint (N + 1 entries), or NULL: grid unaries
    const float *ulam, *uval;
    int grid_len;         // grid unaries: breakpoints 0..grid_len-1, values uval[i * grid_len + l]
    const float *sl, *sr;
    float sl_s, sr_s;
    const float *w, *C;
    float w_s, C_s;
    const int64_t *offsets;
    long long nchains, nnodes;
    int maxlen;
    int T;                // breakpoints a message may hold
    float *x;
    double *energy;
    float2 *arena;        // chain k's M^_i at k * (maxlen + 1) * T, half 1 from ceil(maxlen/2) * T
    int2 *meta;           // per node: (offset in the chain's arena, count)
    float2 *tails;        // per node: end slopes of M^_i
};

__device__ __forceinline__ int chunk_of(int t) { return ((t + WARP - 1) / WARP) | 1; }

// value of the list (P, t; end slopes sl, sr; constant c0 when t == 0) at z, on the
// segment left of index j (P[j-1] <= z <= P[j])
__device__ __forceinline__ float interp_at(const float2 *P, int t, float sl, float sr, float c0,
                                           int j, float z)
{
    if (t == 0) return c0;
    if (j <= 0) return P[0].y + sl * (z - P[0].x);
    if (j >= t) return P[t - 1].y + sr * (z - P[t - 1].x);
    const float2 a = P[j - 1], b = P[j];
    const float d = b.x - a.x;
    return d > 0.f ? a.y + (b.y - a.y) * ((z - a.x) / d) : a.y;
}

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

__device__ __forceinline__ int warp_excl_sum(int v, int lane, int &total)
{
    int inc = v;
#pragma unroll
    for (int o = 1; o < WARP; o <<= 1) {
        const int u = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += u;
    }
    total = __shfl_sync(FULL, inc, WARP - 1);
    return inc - v;
}

// merge A (ta) and B (tb) into O: O = A + B as functions; returns min of O's values (or
// the constant when ta + tb == 0). Ties: A's point first.
__device__ float nc_merge(const float2 *A, int ta, float slA, float srA, float cA, const float2 *B,
                          int tb, float slB, float srB, float2 *O, int lane)
{
    const int t = ta + tb;
    const int per = chunk_of(t);
    const int k0 = min(t, lane * per), k1 = min(t, k0 + per);
    // merge path: i elements of A and k0 - i of B come before output k0
    int lo = max(0, k0 - tb), hi = min(k0, ta);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (A[mid].x <= B[k0 - 1 - mid].x) lo = mid + 1;
        else hi = mid;
    }
    int i = lo, j = k0 - lo;
    float mn = INFINITY;
    for (int k = k0; k < k1; ++k) {
        float2 o;
        if (j >= tb || (i < ta && A[i].x <= B[j].x)) {
            o.x = A[i].x;
            o.y = A[i].y + interp_at(B, tb, slB, srB, 0.f, j, o.x);
            ++i;
        } else {
            o.x = B[j].x;
            o.y = B[j].y + interp_at(A, ta, slA, srA, cA, i, o.x);
            ++j;
        }
        O[k] = o;
        mn = fminf(mn, o.y);
    }
    mn = warp_min(mn);
    return t ? mn : cA;
}

// Algorithm 1 as a scan: O = (H - m) (x) f^1 (REV = false) or (x) f^2 (REV = true), H of
// t points with end slopes sl, sr; values are shifted by -m on the way. With REV the list
// is read from its right end in mirrored coordinates (z -> -z). Optionally copies the
// shifted input to `store` (the record of M^_i). Returns the output count (never above
// t); sets the output's end slopes.
template <bool REV>
__device__ int nc_mc12(const float2 *H, int t, float sl, float sr, float m, float w, float2 *O,
                       float2 *store, int lane, float &osl, float &osr)
{
    // mirrored view: element q of the view is H[REV ? t-1-q : q] at z' = REV ? -x : x
    auto at = [&](int q) -> float2 {
        const float2 e = H[REV ? t - 1 - q : q];
        return make_float2(REV ? -e.x : e.x, e.y - m);
    };
    const float vsl = REV ? -sr : sl, vsr = REV ? -sl : sr;  // end slopes of the view
    const int per = chunk_of(t);
    const int p0 = min(t, lane * per), p1 = min(t, p0 + per);
    if (store) {
        for (int p = p0; p < p1; ++p) {
            const float2 e = H[p];
            store[p] = make_float2(e.x, e.y - m);
        }
    }
    // prefix minimum of g = h - w z over the non-duplicate points (a point equal in z to
    // its predecessor adds nothing)
    float cm = INFINITY;
    for (int q = p0; q < p1; ++q) {
        const float2 e = at(q);
        const bool dup = q > 0 && at(q - 1).x == e.x;
        if (!dup) cm = fminf(cm, fmaf(-w, e.x, e.y));
    }
    float inc = cm;
#pragma unroll
    for (int o = 1; o < WARP; o <<= 1) {
        const float u = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc = fminf(inc, u);
    }
    float excl = __shfl_up_sync(FULL, inc, 1);
    if (lane == 0) excl = INFINITY;
    const float R_all = __shfl_sync(FULL, inc, WARP - 1);
    // count, then write. Point q (not a duplicate): its predecessor pq (the last non-duplicate
    // before it); crossing on (pq, q) iff g_pq > R_pq and g_q < R_pq; point kept iff
    // g_q <= R_{q-1}.
    int pos = 0, total = 0;
    for (int pass = 0; pass < 2; ++pass) {
        float R = excl;  // running minimum over the view's points before q
        float2 prev = make_float2(0.f, 0.f);
        float gprev = INFINITY;
        if (p0 > 0 && p0 < p1) {
            int pq = p0 - 1;
            while (pq > 0 && at(pq - 1).x == at(pq).x) --pq;
            prev = at(pq);
            gprev = fmaf(-w, prev.x, prev.y);
        }
        int c = 0;
        auto emit = [&](float z, float v) {
            if (pass == 1) {
                const int o = REV ? total - 1 - pos - c : pos + c;
                O[o] = make_float2(REV ? -z : z, v);
            }
            ++c;
        };
        for (int q = p0; q < p1; ++q) {
            const float2 e = at(q);
            if (q > 0 && at(q - 1).x == e.x) continue;  // duplicate
            const float g = fmaf(-w, e.x, e.y);
            if (q > 0 && gprev > R && g < R) {
                // the falling segment re-crosses the running minimum
                const float z = prev.x + (e.x - prev.x) * ((R - gprev) / (g - gprev));
                if (z > prev.x && z < e.x) emit(z, fmaf(w, z, R));
            }
            if (g <= R) emit(e.x, e.y);
            R = fminf(R, g);
            prev = e;
            gprev = g;
        }
        // the right end of the view: its last point off the running minimum and g
        // falling there: the end re-crosses the minimum
        if (t > 0 && p1 == t && p0 < p1 && gprev > R_all && vsr < w) {
            const float z = prev.x + (R_all - gprev) / (vsr - w);
            emit(z, fmaf(w, z, R_all));
        }
        if (pass == 0) pos = warp_excl_sum(c, lane, total);
    }
    // end slopes: the left end keeps its slope (<= 0 <= w); the right end follows h where
    // g falls (slope < w), else rises with slope w
    const float nsr = vsr < w ? vsr : w;
    osl = REV ? -nsr : vsl;
    osr = REV ? -vsl : nsr;
    __syncwarp();
    return total;
}

// O = min(H, min H + C) for 0 < C < inf; H has minimum 0 (values relative). End slopes
// become 0. Points whose two neighbouring segments are both flat at the cap are dropped.
// Returns the output count, or -1 (nothing written) if it would exceed `cap_out`.
__device__ int nc_mc3(const float2 *H, int t, float sl, float sr, float C, float2 *O, int cap_out,
                      int lane)
{
    const float cap = C;
    const int per = chunk_of(t);
    const int p0 = min(t, lane * per), p1 = min(t, p0 + per);
    int pos = 0, total = 0;
    for (int pass = 0; pass < 2; ++pass) {
        int c = 0;
        auto emit = [&](float z, float v) {
            if (pass == 1) O[pos + c] = make_float2(z, v);
            ++c;
        };
        for (int p = p0; p < p1; ++p) {
            const float2 e = H[p];
            if (p == 0 && e.y < cap && sl < 0.f) {
                const float z = e.x + (cap - e.y) / sl;
                if (z < e.x) emit(z, cap);
            }
            const bool lflat = p == 0 ? true : H[p - 1].y >= cap;
            const bool rflat = p == t - 1 ? true : H[p + 1].y >= cap;
            if (!(e.y >= cap && lflat && rflat)) emit(e.x, fminf(e.y, cap));
            if (p + 1 < t) {
                const float2 f = H[p + 1];
                const float a = e.y - cap, b = f.y - cap;
                if ((a < 0.f && b > 0.f) || (a > 0.f && b < 0.f)) {
                    const float z = e.x + (f.x - e.x) * (a / (a - b));
                    if (z > e.x && z < f.x) emit(z, cap);
                }
            }
            if (p == t - 1 && e.y < cap && sr > 0.f) {
                const float z = e.x + (cap - e.y) / sr;
                if (z > e.x) emit(z, cap);
            }
        }
        if (pass == 0) {
            pos = warp_excl_sum(c, lane, total);
            if (total > cap_out) return -1;
        }
    }
    __syncwarp();
    return total;
}

struct BestZ {
    float obj;
    int prio;
    float z;
};

__device__ __forceinline__ void best_of(BestZ &b, float obj, int prio, float z)
{
    if (obj < b.obj || (obj == b.obj && prio < b.prio)) b = BestZ{obj, prio, z};
}

__device__ __forceinline__ BestZ warp_best(BestZ b)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(FULL, b.obj, o);
        const int pr = __shfl_xor_sync(FULL, b.prio, o);
        const float z = __shfl_xor_sync(FULL, b.z, o);
        best_of(b, ob, pr, z);
    }
    return b;
}

// argmin over z of H(z) + min(w |xn - z|, C) (pair = true) or of H(z) (pair = false),
// candidates and order as in the file comment; H in global memory.
__device__ float nc_argmin(const float2 *H, int t, float sl, float sr, bool pair, float xn, float w,
                           float C, int lane)
{
    if (t == 0) return pair ? xn : 0.f;
    const int per = chunk_of(t);
    const int p0 = min(t, lane * per), p1 = min(t, p0 + per);
    BestZ b{INFINITY, 0x7fffffff, 0.f};
    const bool trunc = pair && isfinite(C) && w > 0.f;
    const float r = trunc ? C / w : 0.f;
    const float zs[3] = {xn, xn - r, xn + r};
    const int prs[3] = {0, t + 1, t + 2};
    auto pen = [&](float z) {
        if (!pair) return 0.f;
        return fminf(w * fabsf(xn - z), C);
    };
    float2 prevp = make_float2(0.f, 0.f);
    if (p0 > 0 && p0 < p1) prevp = H[p0 - 1];
    for (int p = p0; p < p1; ++p) {
        const float2 e = H[p];
        best_of(b, e.y + pen(e.x), 1 + p, e.x);
        // special candidates on the segment left of p (or the left end)
        if (pair) {
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                if (s > 0 && !trunc) break;
                const float z = zs[s];
                bool in;
                float hz;
                if (p == 0) {
                    in = z < e.x;
                    hz = e.y + sl * (z - e.x);
                } else {
                    in = z >= prevp.x && z < e.x;
                    const float d = e.x - prevp.x;
                    hz = d > 0.f ? prevp.y + (e.y - prevp.y) * ((z - prevp.x) / d) : prevp.y;
                }
                if (in) best_of(b, hz + pen(z), prs[s], z);
            }
        }
        prevp = e;
    }
    if (pair && p1 == t && p0 < p1) {  // right end
        const float2 e = H[t - 1];
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            if (s > 0 && !trunc) break;
            const float z = zs[s];
            if (z >= e.x) best_of(b, e.y + sr * (z - e.x) + pen(z), prs[s], z);
        }
    }
    b = warp_best(b);
    return b.z;
}

// What the two warps of a chain tell each other at the root (shared memory).
struct NcPairXchg {
    double esum[2];   // each half's sum of message minima
    int ta[2], mi[2];  // each half's final message: count, buffer
    float sl[2], sr[2], cA[2];
    int bad[2];
};

__device__ __forceinline__ void pair_bar(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// Two warps per chain, rooted at node mid = n/2 (Algorithm 2 may take any root): warp 0
// of the pair runs the forward pass over nodes 0..mid-1, warp 1 over nodes n-1..mid+1
// (the pairwise terms are symmetric, so the update is the same), each ending with the
// message into the root; after a pair barrier both warps form M^_mid = f_mid + M_L + M_R
// from the two messages and take the same x_mid in argmin M^_mid, then each clips its own
// half outwards. Shared memory per warp: three message buffers of T points.
// At most kNcMaxWarps warps a block; no launch bound, which capped the kernel at 72
// registers and spilled it.
__global__ void nc_chain_kernel(NcArgs p, WsHeader *hdr)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & (WARP - 1);
    const int warp = threadIdx.x / WARP;
    const int role = warp & 1;
    const int pair = warp >> 1;
    const int pairs = blockDim.x / (2 * WARP);
    const long long k = (long long)blockIdx.x * pairs + pair;
    const int T = p.T;
    NcPairXchg *xs = reinterpret_cast<NcPairXchg *>(smem_raw) + pair;
    float2 *buf0 = reinterpret_cast<float2 *>(smem_raw + ((pairs * sizeof(NcPairXchg) + 15) & ~(size_t)15));
    auto Pw = [&](int w, int b) { return buf0 + ((size_t)w * 3 + b) * T; };
    auto P = [&](int b) { return Pw(warp, b); };
    if (k >= p.nchains) return;  // both warps of the pair
    long long start = k * (long long)p.maxlen;
    int n = p.maxlen;
    if (p.offsets) {
        const long long off0 = p.offsets[0], lo = p.offsets[k], hi = p.offsets[k + 1];
        if (lo < off0 || hi < lo || hi - lo > p.maxlen || hi > p.nnodes) {
            if (lane == 0 && role == 0) atomicOr(&hdr->status, ERR_BAD_CHAIN);
            return;
        }
        start = lo;
        n = (int)(hi - lo);
    }
    if (n == 0) {
        if (lane == 0 && role == 0) p.energy[k] = 0.0;
        return;
    }
    const int mid = n >> 1;
    const int cnt = role == 0 ? mid : n - 1 - mid;
    const long long half_cap = (long long)((p.maxlen + 1) / 2) * T;
    float2 *arena = p.arena + k * (long long)(p.maxlen + 1) * T + role * half_cap;
    // node of step j and the node on the root side of its edge
    auto node_of = [&](int j) { return role == 0 ? j : n - 1 - j; };
    auto edge_of = [&](int i) { return role == 0 ? i : i - 1; };  // index of w / C of the edge

    auto load_unary = [&](long long node, float2 *F, int &tf, float &slF, float &srF) -> bool {
        if (p.uoff) {
            const long long u0 = p.uoff[node], u1 = p.uoff[node + 1];
            tf = (int)max(0LL, u1 - u0);
            if (tf > T) return false;
            for (int q = lane; q < tf; q += WARP) F[q] = make_float2(p.ulam[u0 + q], p.uval[u0 + q]);
        } else {
            tf = p.grid_len;
            if (tf > T) return false;
            for (int q = lane; q < tf; q += WARP)
                F[q] = make_float2((float)q, p.uval[node * (long long)p.grid_len + q]);
        }
        slF = p.sl ? p.sl[node] : p.sl_s;
        srF = p.sr ? p.sr[node] : p.sr_s;
        if (tf == 0) slF = srF = 0.f;
        return true;
    };

    // ---------------- forward pass over this warp's half ----------------
    int mi = 0, ta = 0;
    float slA = 0.f, srA = 0.f, cA = 0.f;
    double energy = 0.0;
    unsigned aoff = 0;
    bool bad = false;
    for (int j = 0; j < cnt; ++j) {
        const int i = node_of(j);
        const long long node = start + i;
        const int fi = 1 - mi;
        float2 *F = P(fi);
        int tf;
        float slF, srF;
        if (!load_unary(node, F, tf, slF, srF) || ta + tf > T ||
            (long long)aoff + ta + tf > half_cap) {
            bad = true;
            break;
        }
        __syncwarp();
        float2 *Mh = P(2);
        const int th = ta + tf;
        const float m = nc_merge(P(mi), ta, slA, srA, cA, F, tf, slF, srF, Mh, lane);
        const float slH = slA + slF, srH = srA + srF;
        energy += (double)m;
        __syncwarp();
        if (lane == 0) {
            p.meta[node] = make_int2((int)aoff, th);
            p.tails[node] = make_float2(slH, srH);
        }
        const int e = edge_of(i);
        const float wi = p.w ? p.w[start + e] : p.w_s;
        const float Ci = p.C ? p.C[start + e] : p.C_s;
        // (x) f^1 into F's buffer (free now), recording M^_i; (x) f^2 into mi's buffer
        float s1l, s1r, s2l, s2r;
        const int t1 = nc_mc12<false>(Mh, th, slH, srH, m, wi, F, arena + aoff, lane, s1l, s1r);
        aoff += (unsigned)th;
        const int t2 = nc_mc12<true>(F, t1, s1l, s1r, 0.f, wi, P(mi), nullptr, lane, s2l, s2r);
        if (isfinite(Ci)) {
            if (Ci <= 0.f) {
                ta = 0;
                cA = 0.f;
                slA = srA = 0.f;
            } else {
                const int t3 = nc_mc3(P(mi), t2, s2l, s2r, Ci, F, T, lane);
                if (t3 < 0) {
                    bad = true;
                    break;
                }
                mi = fi;
                ta = t3;
                slA = srA = 0.f;
                cA = 0.f;
            }
        } else {
            ta = t2;
            slA = s2l;
            srA = s2r;
            cA = 0.f;
        }
        __syncwarp();
    }
    bad = __any_sync(FULL, bad);
    if (lane == 0) {
        xs->esum[role] = energy;
        xs->ta[role] = ta;
        xs->mi[role] = mi;
        xs->sl[role] = slA;
        xs->sr[role] = srA;
        xs->cA[role] = cA;
        xs->bad[role] = bad ? 1 : 0;
    }
    pair_bar(1 + pair);

    // ---------------- root: M^_mid = M_L + M_R + f_mid, both warps alike ----------------
    const bool any_bad = xs->bad[0] || xs->bad[1];
    float xmid = 0.f;
    bool root_bad = any_bad;
    int tr = 0;
    float slr = 0.f, srr = 0.f, mr = 0.f;
    if (!any_bad) {
        const int tL = xs->ta[0], tR = xs->ta[1];
        const float2 *ML = Pw(2 * pair, xs->mi[0]), *MR = Pw(2 * pair + 1, xs->mi[1]);
        const int other = 1 - xs->mi[role];  // my free message buffer
        if (tL + tR > T) {
            root_bad = true;
        } else {
            nc_merge(ML, tL, xs->sl[0], xs->sr[0], xs->cA[0], MR, tR, xs->sl[1], xs->sr[1], P(2),
                     lane);
        }
        int tf = 0;
        float slF = 0.f, srF = 0.f;
        if (!root_bad && !load_unary(start + mid, P(other), tf, slF, srF)) root_bad = true;
        if (!root_bad && tL + tR + tf > T) root_bad = true;
        __syncwarp();
        // both warps have read both messages before either overwrites its own
        pair_bar(1 + pair);
        if (!root_bad) {
            const float cLR = (tL + tR == 0) ? xs->cA[0] + xs->cA[1] : 0.f;
            const float slLR = xs->sl[0] + xs->sl[1], srLR = xs->sr[0] + xs->sr[1];
            float2 *R = P(xs->mi[role]);
            mr = nc_merge(P(2), tL + tR, slLR, srLR, cLR, P(other), tf, slF, srF, R, lane);
            tr = tL + tR + tf;
            slr = slLR + slF;
            srr = srLR + srF;
            __syncwarp();
            xmid = nc_argmin(R, tr, slr, srr, false, 0.f, 0.f, 0.f, lane);
        }
    } else {
        pair_bar(1 + pair);
    }
    if (root_bad) {
        if (role == 0) {
            if (lane == 0) {
                atomicOr(&hdr->status, ERR_CAPACITY);
                p.energy[k] = NAN;
            }
            for (int i = lane; i < n; i += WARP) p.x[start + i] = NAN;
        }
        return;
    }
    if (role == 0) {
        if (lane == 0) {
            p.energy[k] = xs->esum[0] + xs->esum[1] + (double)mr;
            p.x[start + mid] = xmid;
        }
    }
    __syncwarp();
    __threadfence_block();
    // ---------------- backward: clip this half outwards from the root ----------------
    float xn = xmid;
    for (int j = cnt - 1; j >= 0; --j) {
        const int i = node_of(j);
        const long long node = start + i;
        const int2 mt = p.meta[node];
        const float2 tl = p.tails[node];
        const int e = edge_of(i);
        const float wi = p.w ? p.w[start + e] : p.w_s;
        const float Ci = p.C ? p.C[start + e] : p.C_s;
        const float xi = nc_argmin(arena + mt.x, mt.y, tl.x, tl.y, true, xn, wi, Ci, lane);
        if (lane == 0) p.x[node] = xi;
        xn = xi;
    }
}

struct NcWs {
    WsHeader *hdr;
    float2 *arena;
    int2 *meta;
    float2 *tails;
    size_t bytes;
};

NcWs carve_nc(void *base, long long nodes, long long nchains, long long maxlen, int T)
{
    Carver cv(base);
    NcWs o;
    o.hdr = cv.take<WsHeader>(1);
    o.meta = cv.take<int2>((size_t)nodes);
    o.tails = cv.take<float2>((size_t)nodes);
    o.arena = cv.take<float2>((size_t)(nchains * (maxlen + 1) * (long long)T));
    o.bytes = align_up(cv.used, 256);
    return o;
}

}  // namespace

extern "C" {

size_t tv_chain_nonconvex_workspace_size(int64_t num_nodes, int64_t num_chains, int64_t max_len,
                                         int max_breakpoints)
{
    if (num_nodes < 0 || num_chains < 0 || max_len < 0 || max_breakpoints < 1) return 0;
    return carve_nc(nullptr, num_nodes, num_chains, max_len, max_breakpoints).bytes;
}

tv_status tv_chain_solve_nonconvex(const int64_t *d_uoff, const float *d_ulam,
                                   const float *d_uval, int grid_len, const float *d_sl,
                                   const float *d_sr, float sl, float sr, const float *d_w,
                                   float w, const float *d_C, float C, const int64_t *d_offsets,
                                   int64_t num_nodes, int64_t num_chains, int64_t max_len,
                                   int max_breakpoints, float *d_x, double *d_energy,
                                   void *d_workspace, size_t workspace_bytes, tv_stream_t stream)
{
    clear_error();
    if (num_chains < 0 || max_len < 0 || num_nodes < 0 || max_breakpoints < 1 ||
        max_breakpoints > 4096 || max_len > (1LL << 24)) {
        set_error("tv_chain_solve_nonconvex: need num_chains, max_len, num_nodes >= 0 and "
                  "1 <= max_breakpoints <= 4096");
        return TV_ERR_INVALID;
    }
    if (max_len * (long long)max_breakpoints >= (1LL << 31)) {
        set_error("tv_chain_solve_nonconvex: max_len * max_breakpoints must stay below 2^31");
        return TV_ERR_INVALID;
    }
    if (!d_offsets && num_nodes != num_chains * max_len) {
        set_error("tv_chain_solve_nonconvex: without offsets, num_nodes = num_chains * max_len");
        return TV_ERR_INVALID;
    }
    if (!d_uval || !d_x || !d_energy || !d_workspace || (d_uoff && !d_ulam) ||
        (!d_uoff && grid_len < 1)) {
        set_error("tv_chain_solve_nonconvex: uval, x, energy and workspace must not be NULL; "
                  "ulam with uoff, or grid_len >= 1 without");
        return TV_ERR_INVALID;
    }
    if (!d_uoff && grid_len > max_breakpoints) {
        set_error("tv_chain_solve_nonconvex: grid_len above max_breakpoints");
        return TV_ERR_INVALID;
    }
    if ((!d_sl && !(sl <= 0.f)) || (!d_sr && !(sr >= 0.f)) ||
        (!d_w && !(w >= 0.f && w < INFINITY)) || (!d_C && !(C >= 0.f))) {
        set_error("tv_chain_solve_nonconvex: need sl <= 0 <= sr, finite w >= 0, C >= 0");
        return TV_ERR_INVALID;
    }
    if (num_chains == 0 || max_len == 0) return TV_OK;
    NcWs ws = carve_nc(d_workspace, num_nodes, num_chains, max_len, max_breakpoints);
    if (workspace_bytes < ws.bytes) {
        set_error("tv_chain_solve_nonconvex: workspace of %zu bytes, %zu needed", workspace_bytes,
                  ws.bytes);
        return TV_ERR_NOMEM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    tv_status st = check_cuda(cudaMemsetAsync(ws.hdr, 0, sizeof(WsHeader), s), "memset");
    if (st != TV_OK) return st;
    NcArgs p{d_uoff, d_ulam, d_uval, grid_len, d_sl, d_sr, sl, sr, d_w, d_C, w, C, d_offsets,
             num_chains, num_nodes, (int)max_len, max_breakpoints, d_x, d_energy, ws.arena,
             ws.meta, ws.tails};
    const int pairs = std::max(1, nc_warps(max_breakpoints) / 2);
    const int wpb = 2 * pairs;
    const size_t smem = ((pairs * sizeof(NcPairXchg) + 15) & ~(size_t)15) +
                        (size_t)wpb * 3 * max_breakpoints * sizeof(float2);
    st = check_cuda(cudaFuncSetAttribute(nc_chain_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    "cudaFuncSetAttribute");
    if (st != TV_OK) return st;
    const long long blocks = (num_chains + pairs - 1) / pairs;
    const bool prof = prof_on();
    if (prof) prof_mark(PK_CHAIN, s, true);
    nc_chain_kernel<<<(unsigned)blocks, wpb * WARP, smem, s>>>(p, ws.hdr);
    st = check_cuda(cudaGetLastError(), "non-convex chain kernel launch");
    if (st == TV_OK) note_launch();
    if (prof) prof_mark(PK_CHAIN, s, false);
    return st;
}

}  // extern "C"
