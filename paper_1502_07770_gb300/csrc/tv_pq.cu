// Chains with piecewise-quadratic unaries (Sec. 4.2):
//     x* = argmin_x sum_i (a_i x_i^2 / 2 - b_i x_i + alpha_i |x_i - f_i|) + sum_{i<n} w_i |x_{i+1} - x_i|,
// the convex chain of Algorithm 2 whose unary derivatives g_i(z) = a_i z - b_i +
// alpha_i sign(z - f_i) are piecewise linear with a jump of 2 alpha_i at f_i. It is the
// row proximal map of TV-l1 denoising (Sec. 6): alpha = 1, a = 1/tau, b = xi/tau, or,
// multiplied through by tau, a = 1, b = xi, alpha = tau (the form tv2d_denoise_l1 uses).
//
// One warp per chain. The message (a derivative) is held in registers, one breakpoint
// per lane: its position lambda_k, the message's left and right limits L_k <= R_k there
// (a jump where they differ) and its slope S_k on the piece to the right (0 right of the
// last breakpoint); left of the first breakpoint it is constant at its left bound. Per
// node: f_i is inserted (a ballot finds its place, one shuffle opens the slot), z - ... is
// added to every limit (a_i lambda_k - b_i, -alpha_i left of f_i and +alpha_i right of it,
// the jump 2 alpha_i at f_i), a_i to every slope; then the clip to [-w_i, w_i] finds
//   lambda^- = sup{z : m^_i(z) < -w_i},  lambda^+ = inf{z : m^_i(z) > w_i}
// either inside a piece (every lane computes its piece's crossings) or at a jump.
// Backward: x_i = clip(x_{i+1}, lambda^-_i, lambda^+_i), 32 clips composed per step.
// A message of more than 32 breakpoints is finished by lane 0 from global memory.
#include <cuda_runtime.h>

#include <atomic>

#include "tv_launch.cuh"

using namespace tvk;
using namespace tvh;

namespace {

__device__ __forceinline__ float warp_min_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

__device__ __forceinline__ float warp_max_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

struct PqState {
    float lam, L, R, S;  // this lane's breakpoint
    int size;
    float lam0, L0;      // the first breakpoint and its left limit (every lane)
    float wlo_p;         // the message's value left of its first breakpoint
};

// One node: returns the clip points; sets ovf (sticky) if more than 32 breakpoints
// would be needed (the state is then meaningless).
__device__ __forceinline__ void pq_update(PqState &s, float a, float b, float al, float f,
                                          float wlo, float whi, int lane, bool &ovf, float &lm,
                                          float &hp)
{
    bool valid = lane < s.size;
    // ---- insert f (unless a breakpoint is already there) ----
    const unsigned below = __ballot_sync(FULL, valid && s.lam < f);
    const int ins = __popc(below);
    const float lam_at = __shfl_sync(FULL, s.lam, ins & 31);
    const bool exists = ins < s.size && lam_at == f;
    if (!exists) {
        if (s.size + 1 > WARP) ovf = true;
        const int src = (ins - 1) & 31;
        const float pl = __shfl_sync(FULL, s.lam, src), pR = __shfl_sync(FULL, s.R, src),
                    pS = __shfl_sync(FULL, s.S, src);
        float mval, Sn;
        if (ins == 0) {
            mval = s.size > 0 ? s.wlo_p : 0.f;  // the message's flat left end (0 before node 0)
            Sn = 0.f;
        } else {
            mval = fmaf(pS, f - pl, pR);
            Sn = pS;
        }
        const float ul = __shfl_up_sync(FULL, s.lam, 1), uL = __shfl_up_sync(FULL, s.L, 1),
                    uR = __shfl_up_sync(FULL, s.R, 1), uS = __shfl_up_sync(FULL, s.S, 1);
        if (lane == ins) {
            s.lam = f;
            s.L = mval;
            s.R = mval;
            s.S = Sn;
        } else if (lane > ins) {
            s.lam = ul;
            s.L = uL;
            s.R = uR;
            s.S = uS;
        }
        s.size += 1;
        valid = lane < s.size;
    }
    // ---- transformation (a): + a z - b - alpha left of f, + alpha right of it ----
    {
        const float lin = fmaf(a, s.lam, -b);
        const float dl = (lane <= ins) ? -al : al;
        const float dr = (lane < ins) ? -al : al;
        s.L += lin + dl;
        s.R += lin + dr;
        s.S += a;
    }
    const float lam_n = __shfl_down_sync(FULL, s.lam, 1);
    const bool last = lane == s.size - 1;
    // crossings of wlo and whi on the piece right of this breakpoint (the last piece has
    // slope a), clamped to the piece
    float cL = fmaxf(s.lam + __fdividef(wlo - s.R, s.S), s.lam);
    float cR = fmaxf(s.lam + __fdividef(whi - s.R, s.S), s.lam);
    if (!last) {
        cL = fminf(cL, lam_n);
        cR = fminf(cR, lam_n);
    }
    const unsigned bge = __ballot_sync(FULL, valid && s.R >= wlo);
    const unsigned ble = __ballot_sync(FULL, valid && s.L <= whi);
    // trailing zeros of an empty vote are 32 (ell = size); 31 - clz(0) = -1 (no kept point)
    const int ell = min(__clz(__brev(bge)), s.size);
    const int kl = 31 - __clz(ble);
    const float L0 = __shfl_sync(FULL, s.L, 0), lam0 = __shfl_sync(FULL, s.lam, 0);
    const float Le = __shfl_sync(FULL, s.L, ell & 31), Re = __shfl_sync(FULL, s.R, ell & 31),
                lame = __shfl_sync(FULL, s.lam, ell & 31), Se = __shfl_sync(FULL, s.S, ell & 31);
    const float cLm = __shfl_sync(FULL, cL, (ell - 1) & 31), Sm = __shfl_sync(FULL, s.S, (ell - 1) & 31);
    const float Lk = __shfl_sync(FULL, s.L, kl & 31), Rk = __shfl_sync(FULL, s.R, kl & 31),
                lamk = __shfl_sync(FULL, s.lam, kl & 31), cRk = __shfl_sync(FULL, cR, kl & 31);
    const bool jumpL = ell < s.size && Le < wlo;
    const bool jumpR = kl >= 0 && Rk > whi;
    const bool both = jumpL && jumpR && ell == kl;
    float Sl;
    if (jumpL) {
        lm = lame;
        Sl = Se;
    } else if (ell == 0) {
        lm = fminf(lam0 + (wlo - L0) / a, lam0);  // on the left end piece (slope a)
        Sl = a;
    } else {
        lm = cLm;
        Sl = Sm;
    }
    if (jumpR) hp = lamk;
    else if (kl < 0) hp = fminf(lam0 + (whi - L0) / a, lam0);
    else hp = cRk;
    const int k0 = ell + (jumpL ? 1 : 0), k1 = kl - (jumpR ? 1 : 0);
    const int K = k1 >= k0 ? k1 - k0 + 1 : 0;
    if (K + 2 > WARP) ovf = true;
    const float lmR = jumpL ? fminf(Re, whi) : wlo;
    const float hpL = jumpR ? (both ? fminf(Re, whi) : fmaxf(Lk, wlo)) : whi;
    const int src = (lane - 1 + k0) & 31;
    const float nl = __shfl_sync(FULL, s.lam, src), nL = __shfl_sync(FULL, s.L, src),
                nR = __shfl_sync(FULL, s.R, src), nS = __shfl_sync(FULL, s.S, src);
    if (lane == 0) {
        s.lam = lm;
        s.L = wlo;
        s.R = lmR;
        s.S = both ? 0.f : Sl;
    } else if (lane == K + 1) {
        s.lam = hp;
        s.L = hpL;
        s.R = whi;
        s.S = 0.f;
    } else {
        s.lam = nl;
        s.L = nL;
        s.R = nR;
        s.S = nS;
    }
    s.size = K + 2;
    s.wlo_p = wlo;
}

// pq_update for a 16-lane half (two chain halves per warp), in ring form: the breakpoints
// sit at ring positions 0 .. size-1 counted from a head lane, each lane carrying its
// position idx. Inserting f
// at position ins moves the entries at positions ins.. up by one (one fixed-offset
// shuffle per field: every lane reads its ring predecessor, which for the new entry is
// also the entry the message's value at f is read from). Removing entries at either end
// moves nothing: lambda^- and lambda^+ take the lanes of the entries they replace (the
// last one removed on the left, the first one removed on the right, or the entry at a
// jump itself), and the positions shift. The counts that place them are population
// counts of votes (limits increase along the ring): entries with R < w^-, with L <= w^+,
// and the jumps from those with L < w^- and with R <= w^+. The lanes that take lambda^-
// and lambda^+ store the step's record. The arithmetic is pq_update's.
struct PqRing {
    float lam, L, R, S;  // this lane's entry (ring position idx)
    int idx, size;
    float wlo_p;         // the message's value left of its first breakpoint
};

template <bool ALWAYS>
__device__ __forceinline__ void pq_ring_update(PqRing &s, float a, float b, float al, float f,
                                               float wlo, float whi, int sl, unsigned seg_mask,
                                               bool active, bool &ovf, float2 *rec)
{
    constexpr int G = 16;
    const int prv = (sl - 1) & (G - 1), nxt = (sl + 1) & (G - 1);
    bool valid = s.idx < s.size;
    // ---- insert f (unless an entry is already there) ----
    const int ins = __popc(__ballot_sync(FULL, valid && s.lam < f) & seg_mask);
    const bool fresh = (__ballot_sync(FULL, valid && s.lam == f) & seg_mask) == 0u;
    const float ul = __shfl_sync(FULL, s.lam, prv, G), uL = __shfl_sync(FULL, s.L, prv, G),
                uR = __shfl_sync(FULL, s.R, prv, G), uS = __shfl_sync(FULL, s.S, prv, G);
    if (ALWAYS || active) {
        if (fresh && s.size + 1 > G) ovf = true;
        const bool at = fresh && s.idx == ins;
        const bool up = fresh && s.idx > ins && s.idx <= s.size;
        const float mval = ins == 0 ? (s.size > 0 ? s.wlo_p : 0.f) : fmaf(uS, f - ul, uR);
        const float Sn = ins == 0 ? 0.f : uS;
        s.lam = at ? f : (up ? ul : s.lam);
        s.L = at ? mval : (up ? uL : s.L);
        s.R = at ? mval : (up ? uR : s.R);
        s.S = at ? Sn : (up ? uS : s.S);
        s.size += fresh ? 1 : 0;
        // ---- transformation (a): + a z - b - alpha left of f, + alpha right of it ----
        const float lin = fmaf(a, s.lam, -b);
        s.L += lin + (s.idx <= ins ? -al : al);
        s.R += lin + (s.idx < ins ? -al : al);
        s.S += a;
    }
    valid = s.idx < s.size;
    const float lam_n = __shfl_sync(FULL, s.lam, nxt, G), R_n = __shfl_sync(FULL, s.R, nxt, G);
    const bool last = s.idx == s.size - 1;
    float cL = fmaxf(s.lam + __fdividef(wlo - s.R, s.S), s.lam);
    float cR = fmaxf(s.lam + __fdividef(whi - s.R, s.S), s.lam);
    if (!last) {
        cL = fminf(cL, lam_n);
        cR = fminf(cR, lam_n);
    }
    const float cR_prev = __shfl_sync(FULL, cR, prv, G);
    const int head = (sl - s.idx) & (G - 1);
    const float lam0 = __shfl_sync(FULL, s.lam, head, G), L0 = __shfl_sync(FULL, s.L, head, G);
    const int ell = __popc(__ballot_sync(FULL, valid && s.R < wlo) & seg_mask);
    const int kl = __popc(__ballot_sync(FULL, valid && s.L <= whi) & seg_mask) - 1;
    const bool jumpL = __popc(__ballot_sync(FULL, valid && s.L < wlo) & seg_mask) > ell;
    const bool jumpR = __popc(__ballot_sync(FULL, valid && s.R <= whi) & seg_mask) <= kl;
    const bool both = jumpL && jumpR && ell == kl;
    const int k0 = ell + (jumpL ? 1 : 0), k1 = kl - (jumpR ? 1 : 0);
    const int K = k1 >= k0 ? k1 - k0 + 1 : 0;
    if ((ALWAYS || active) && K + 2 > G) ovf = true;
    if (ALWAYS || active) {
        const int p_lm = (jumpL && !both) ? ell : ell - 1;  // ring position of lambda^-
        const int p_hp = jumpR ? kl : kl + 1;               // of lambda^+
        const bool is_lm = s.idx == (p_lm & (G - 1)), is_hp = s.idx == (p_hp & (G - 1));
        const float lm_end = fminf(lam0 + (wlo - L0) / a, lam0);  // on the left end piece
        const float hp_end = fminf(lam0 + (whi - L0) / a, lam0);
        const float lmv = both ? lam_n : (jumpL ? s.lam : (ell == 0 ? lm_end : cL));
        const float lmR = both ? fminf(R_n, whi) : (jumpL ? fminf(s.R, whi) : wlo);
        const float lmS = both ? 0.f : (jumpL ? s.S : (ell == 0 ? a : s.S));
        const float hpv = jumpR ? s.lam : (kl < 0 ? hp_end : cR_prev);
        const float hpL = both ? fminf(s.R, whi) : (jumpR ? fmaxf(s.L, wlo) : whi);
        if (is_lm) rec->x = lmv;
        if (is_hp) rec->y = hpv;
        s.lam = is_lm ? lmv : (is_hp ? hpv : s.lam);
        s.L = is_lm ? wlo : (is_hp ? hpL : s.L);
        s.R = is_lm ? lmR : (is_hp ? whi : s.R);
        s.S = is_lm ? lmS : (is_hp ? 0.f : s.S);
        s.idx = (s.idx - p_lm) & (G - 1);
        s.size = K + 2;
        s.wlo_p = wlo;
    }
}

// Overflow path: lane 0, the same update on a global array of (lambda, L, R, S) entries
// (4 * (3n + 4) floats), sequential and O(size) per node.
struct PqEntry {
    float lam, L, R, S;
};

__device__ void pq_lane0(int n, const float *a, const float *b, const float *al, const float *f,
                         const float *w, float wscale, float alpha, float lam, float *x,
                         PqEntry *E, PqEntry *Etmp, float2 *rec)
{
    int size = 0;
    float wlo_p = 0.f;
    for (int i = 0; i < n; ++i) {
        const float ai = a ? a[i] : 1.f, bi = b[i], ali = al ? al[i] : alpha, fi = f[i];
        const float wi = (i < n - 1) ? (w ? w[i] * wscale : lam) : 0.f;
        const float wlo = -wi, whi = wi;
        int ins = 0;
        while (ins < size && E[ins].lam < fi) ++ins;
        const bool exists = ins < size && E[ins].lam == fi;
        if (!exists) {
            float mval = 0.f, Sn = 0.f;
            if (ins == 0) mval = size > 0 ? wlo_p : 0.f;
            else {
                mval = fmaf(E[ins - 1].S, fi - E[ins - 1].lam, E[ins - 1].R);
                Sn = E[ins - 1].S;
            }
            for (int q = size; q > ins; --q) E[q] = E[q - 1];
            E[ins] = PqEntry{fi, mval, mval, Sn};
            ++size;
        }
        for (int k = 0; k < size; ++k) {
            const float lin = fmaf(ai, E[k].lam, -bi);
            E[k].L += lin + (k <= ins ? -ali : ali);
            E[k].R += lin + (k < ins ? -ali : ali);
            E[k].S += ai;
        }
        int ell = size, kl = -1;
        for (int k = 0; k < size; ++k)
            if (E[k].R >= wlo) {
                ell = k;
                break;
            }
        for (int k = size - 1; k >= 0; --k)
            if (E[k].L <= whi) {
                kl = k;
                break;
            }
        auto cross = [&](int k, float lev) {
            float z = fmaxf(E[k].lam + (lev - E[k].R) / E[k].S, E[k].lam);
            if (k < size - 1) z = fminf(z, E[k + 1].lam);
            return z;
        };
        const bool jumpL = ell < size && E[ell].L < wlo;
        const bool jumpR = kl >= 0 && E[kl].R > whi;
        const bool both = jumpL && jumpR && ell == kl;
        float lm, hp, Sl;
        if (jumpL) {
            lm = E[ell].lam;
            Sl = E[ell].S;
        } else if (ell == 0) {
            lm = fminf(E[0].lam + (wlo - E[0].L) / ai, E[0].lam);
            Sl = ai;
        } else {
            lm = cross(ell - 1, wlo);
            Sl = E[ell - 1].S;
        }
        if (jumpR) hp = E[kl].lam;
        else if (kl < 0) hp = fminf(E[0].lam + (whi - E[0].L) / ai, E[0].lam);
        else hp = cross(kl, whi);
        const int k0 = ell + (jumpL ? 1 : 0), k1 = kl - (jumpR ? 1 : 0);
        int nt = 0;
        Etmp[nt++] = PqEntry{lm, wlo, jumpL ? fminf(E[ell].R, whi) : wlo, both ? 0.f : Sl};
        for (int k = k0; k <= k1; ++k) Etmp[nt++] = E[k];
        Etmp[nt++] = PqEntry{hp, jumpR ? (both ? fminf(E[ell].R, whi) : fmaxf(E[kl].L, wlo)) : whi,
                             whi, 0.f};
        for (int q = 0; q < nt; ++q) E[q] = Etmp[q];
        size = nt;
        wlo_p = wlo;
        rec[i] = make_float2(lm, hp);
    }
    float xv = 0.5f * (rec[n - 1].x + rec[n - 1].y);
    x[n - 1] = xv;
    for (int i = n - 2; i >= 0; --i) {
        xv = clip_to(xv, rec[i].x, rec[i].y);
        x[i] = xv;
    }
}

struct PqArgs {
    const float *a, *b, *al, *f, *w;
    float alpha, lam;  // used where al / w are NULL
    float wscale;      // multiplies every edge weight
    long long w_stride;  // > 0: chain k's weights at w + k * w_stride (image rows), else w + start
    const int64_t *offsets;
    long long nchains;
    int maxlen;
    float *x;
    float2 *rec;    // records: chain k at k * maxlen
    PqEntry *ent;   // overflow entries: chain k at k * 2 * (3 maxlen + 4)
};

constexpr int kPqWarps = 4;

// Chain k (first node `start`, n nodes) by the calling warp from node 0: the 32-lane
// update, records, backward clips; lane 0 from the workspace past 32 breakpoints.
__device__ void pq_solve_warp(const PqArgs &p, long long k, long long start, int n, int lane,
                              WsHeader *hdr)
{
    float2 *rec = p.rec + k * (long long)p.maxlen;
    const float *a = p.a ? p.a + start : nullptr;
    const float *b = p.b + start, *f = p.f + start;
    const float *al = p.al ? p.al + start : nullptr;
    const float *w = p.w ? p.w + (p.w_stride > 0 ? k * p.w_stride : start) : nullptr;
    PqState s{0.f, 0.f, 0.f, 0.f, 0, 0.f, 0.f, 0.f};
    bool ovf = false;
    float xlast = 0.f;
    const int nblocks = (n + WARP - 1) / WARP;
    for (int blk = 0; blk < nblocks && !ovf; ++blk) {
        const int i_l = blk * WARP + lane;
        const bool in = i_l < n;
        const float av = (in && a) ? a[i_l] : 1.f, bv = in ? b[i_l] : 0.f,
                    alv = in ? (al ? al[i_l] : p.alpha) : 0.f, fv = in ? f[i_l] : 0.f,
                    wv = (i_l < n - 1) ? (w ? w[i_l] * p.wscale : p.lam) : 0.f;
        const int cnt = min(WARP, n - blk * WARP);
        for (int j = 0; j < cnt; ++j) {
            const int i = blk * WARP + j;
            const float ai = __shfl_sync(FULL, av, j), bi = __shfl_sync(FULL, bv, j),
                        ali = __shfl_sync(FULL, alv, j), fi = __shfl_sync(FULL, fv, j),
                        wi = __shfl_sync(FULL, wv, j);
            float lm, hp;
            pq_update(s, ai, bi, ali, fi, -wi, wi, lane, ovf, lm, hp);
            if (i == n - 1) xlast = 0.5f * (lm + hp);
            else if (lane == 0) rec[i] = make_float2(lm, hp);
        }
        ovf = __any_sync(FULL, ovf);
    }
    __syncwarp();
    if (ovf) {
        if (lane == 0) {
            atomicAdd(&hdr->overflowed, 1ull);
            PqEntry *E = p.ent + k * 2LL * (3LL * p.maxlen + 4);
            pq_lane0(n, a, b, al, f, w, p.wscale, p.alpha, p.lam, p.x + start, E,
                     E + (3LL * p.maxlen + 4), rec);
        }
        return;
    }
    float x_next = xlast;
    for (int blk = nblocks - 1; blk >= 0; --blk) {
        const int i = blk * WARP + lane;
        float lo = -INFINITY, hi = INFINITY;
        if (i < n - 1) {
            const float2 r = rec[i];
            lo = r.x;
            hi = r.y;
        }
        const float xv = clip_suffix(lo, hi, x_next, lane, min(WARP, n - blk * WARP));
        if (i < n) p.x[start + i] = xv;
        x_next = __shfl_sync(FULL, xv, 0);
    }
}

// chain offsets: chain k's first node and length (false: malformed, flagged)
__device__ __forceinline__ bool pq_chain_of(const PqArgs &p, long long k, int lane, WsHeader *hdr,
                                            long long &start, int &n)
{
    start = k * (long long)p.maxlen;
    n = p.maxlen;
    if (p.offsets) {
        const long long off0 = p.offsets[0], lo = p.offsets[k], hi = p.offsets[k + 1];
        if (lo < off0 || hi < lo || hi - lo > p.maxlen) {
            if (lane == 0) atomicOr(&hdr->status, ERR_BAD_CHAIN);
            return false;
        }
        start = lo;
        n = (int)(hi - lo);
    }
    return true;
}

__global__ void __launch_bounds__(kPqWarps * WARP) pq_chain_kernel(PqArgs p, WsHeader *hdr)
{
    pdl_enter();
    const int lane = threadIdx.x & (WARP - 1);
    const long long k = (long long)blockIdx.x * kPqWarps + threadIdx.x / WARP;
    if (k >= p.nchains) return;
    long long start;
    int n;
    if (!pq_chain_of(p, k, lane, hdr, start, n) || n == 0) return;
    pq_solve_warp(p, k, start, n, lane, hdr);
}

// ------------------------------------------------------ middle-rooted chains --
// Rooted at node mid = n/2 (Algorithm 2 allows any root), a chain's two halves each end
// with the message into the root; the root x_mid is the zero of
//     g(z) = a z - b + alpha sign(z - f) + m_L(z) + m_R(z)
// (non-decreasing, piecewise linear with jumps): every breakpoint of either message and
// f are candidates; the first candidate c1 with g(c1+) >= 0 is the root if g(c1-) <= 0,
// else the root lies on the linear piece between c1 and the candidate c0 before it.
struct PqMsg {
    float lam[WARP], L[WARP], R[WARP], S[WARP];
    int size, ovf;
};

// value of message M just left (m_lo) and right (m_hi) of z, and its slope right of z
__device__ __forceinline__ void pq_msg_at(const PqMsg &M, float z, float &m_lo, float &m_hi,
                                          float &slope)
{
    const int t = M.size;
    if (t == 0) {
        m_lo = m_hi = slope = 0.f;
        return;
    }
    // e = entries with lam <= z, j = entries with lam < z
    int e = 0, j = 0;
    for (int q = 0; q < t; ++q) {
        e += M.lam[q] <= z;
        j += M.lam[q] < z;
    }
    if (e == 0) {
        m_hi = M.L[0];
        slope = 0.f;
    } else {
        const int q = e - 1;
        m_hi = M.lam[q] == z ? M.R[q] : fmaf(M.S[q], z - M.lam[q], M.R[q]);
        slope = M.S[q];
    }
    if (j < t && M.lam[j] == z) m_lo = M.L[j];
    else if (j == 0) m_lo = M.L[0];
    else m_lo = fmaf(M.S[j - 1], z - M.lam[j - 1], M.R[j - 1]);
}

__device__ float pq_root(const PqMsg &ML, const PqMsg &MR, float a, float b, float al, float f,
                         int lane)
{
    float cand[3];
    int nc = 0;
    if (lane < ML.size) cand[nc++] = ML.lam[lane];
    if (lane < MR.size) cand[nc++] = MR.lam[lane];
    if (lane == 0) cand[nc++] = f;
    float gm[3], gp[3], sp[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        gm[q] = gp[q] = sp[q] = 0.f;
        if (q < nc) {
            const float c = cand[q];
            float l1, h1, s1, l2, h2, s2;
            pq_msg_at(ML, c, l1, h1, s1);
            pq_msg_at(MR, c, l2, h2, s2);
            const float lin = fmaf(a, c, -b);
            gm[q] = lin + (c <= f ? -al : al) + l1 + l2;
            gp[q] = lin + (c < f ? -al : al) + h1 + h2;
            sp[q] = a + s1 + s2;
        }
    }
    float c1 = INFINITY;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        if (q < nc && gp[q] >= 0.f) c1 = fminf(c1, cand[q]);
    c1 = warp_min_f(c1);
    const float lEndL = ML.size ? ML.L[0] : 0.f, lEndR = MR.size ? MR.L[0] : 0.f;
    if (!(c1 < INFINITY)) {
        // right of every candidate: both messages at their right ends
        const float rL = ML.size ? ML.R[ML.size - 1] : 0.f, rR = MR.size ? MR.R[MR.size - 1] : 0.f;
        return (b - al - rL - rR) / a;
    }
    float g1m = -INFINITY, c0 = -INFINITY;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (q < nc && cand[q] == c1) g1m = fmaxf(g1m, gm[q]);
        if (q < nc && cand[q] < c1) c0 = fmaxf(c0, cand[q]);
    }
    g1m = warp_max_f(g1m);
    if (g1m <= 0.f) return c1;  // a jump of g (or an exact zero) at c1
    c0 = warp_max_f(c0);
    if (!(c0 > -INFINITY)) {
        // left of every candidate: both messages at their left ends, the unary at -alpha
        return fminf((b + al - lEndL - lEndR) / a, c1);
    }
    float g0 = -INFINITY, s0 = -INFINITY;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        if (q < nc && cand[q] == c0) {
            g0 = fmaxf(g0, gp[q]);
            s0 = fmaxf(s0, sp[q]);
        }
    g0 = warp_max_f(g0);
    s0 = warp_max_f(s0);
    const float z = c0 - g0 / s0;
    return fminf(fmaxf(z, c0), c1);
}

// ----------------------------------------------------- middle-rooted halves --
// One warp per chain, rooted at node mid = n/2: lanes 0-15 run pq_ring_update over
// nodes 0..mid-1, lanes 16-31 over nodes n-1..mid+1, both in the same instructions;
// the two messages into the root (at most 16 breakpoints each) go to shared memory and
// the whole warp finds the root (pq_root), then each segment clips its
// half outwards. A half that outgrows 16 breakpoints sends the chain to the one-warp
// solve from node 0 (32 breakpoints, then lane 0 from the workspace).
// Up to 16 update steps of both halves (positions base..base+15; c16 of them exist).
// ALWAYS: every step is an update in both halves. U: curvature 1, one alpha and one
// weight for the whole chain, so only b and f are shuffled.
template <bool ALWAYS, bool U>
__device__ __forceinline__ void pq_half_steps(PqRing &s, bool &ovf, float2 *rec, int base,
                                              int c16, int cnt, int n, int seg, int sl,
                                              int seg_shift, float av, float bv, float alv,
                                              float fv, float wv, float alpha, float lam)
{
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
        if (!ALWAYS && jj >= c16) break;  // c16 is the same in every lane
        const float bi = __shfl_sync(FULL, bv, jj, 16), fi = __shfl_sync(FULL, fv, jj, 16);
        float ai = 1.f, ali = alpha, wi = lam;
        if constexpr (!U) {
            ai = __shfl_sync(FULL, av, jj, 16);
            ali = __shfl_sync(FULL, alv, jj, 16);
            wi = __shfl_sync(FULL, wv, jj, 16);
        }
        const int q = base + jj;
        const bool active = ALWAYS || q < cnt;
        pq_ring_update<ALWAYS>(s, ai, bi, ali, fi, -wi, wi, sl, 0xFFFFu << seg_shift, active, ovf,
                               rec + (seg == 0 ? q : n - 1 - q));
    }
}

// This lane's node of block blk of its half (the inputs of a block are loaded one block
// ahead): node j of the left half is j, of the right half n-1-j, whose edge towards the
// root is the one before it.
template <bool U>
__device__ __forceinline__ void pq_half_load(const PqArgs &p, const float *a, const float *b,
                                             const float *al, const float *f, const float *w,
                                             int blk, int sl, int seg, int n, int cnt, float &av,
                                             float &bv, float &alv, float &fv, float &wv)
{
    const int j_l = blk * 16 + sl;
    const bool in = j_l < cnt;
    const int i_l = in ? (seg == 0 ? j_l : n - 1 - j_l) : 0;
    bv = in ? b[i_l] : 0.f;
    fv = in ? f[i_l] : 0.f;
    if constexpr (U) {
        av = 1.f;
        alv = p.alpha;
        wv = p.lam;
    } else {
        const int e_l = seg == 0 ? i_l : i_l - 1;
        av = (in && a) ? a[i_l] : 1.f;
        alv = in ? (al ? al[i_l] : p.alpha) : 0.f;
        wv = in ? (w ? w[e_l] * p.wscale : p.lam) : 0.f;
    }
}

// Launched with kPqWarps warps per block and no launch bound (a bound capped the
// kernel at 72 registers and spilled the update). U: see pq_half_steps.
template <bool U>
__global__ void pq_halves_kernel(PqArgs p, WsHeader *hdr)
{
    pdl_enter();
    __shared__ PqMsg msg[kPqWarps][2];
    const int lane = threadIdx.x & (WARP - 1);
    const int warp = threadIdx.x / WARP;
    const long long k = (long long)blockIdx.x * kPqWarps + warp;
    if (k >= p.nchains) return;
    long long start;
    int n;
    if (!pq_chain_of(p, k, lane, hdr, start, n) || n == 0) return;
    const int mid = n >> 1;
    const int seg = lane >> 4, sl = lane & 15, seg_shift = seg * 16;
    const int cnt = seg == 0 ? mid : n - 1 - mid;
    const int cmax = max(mid, n - 1 - mid);
    auto node_of = [&](int j) { return seg == 0 ? j : n - 1 - j; };
    float2 *rec = p.rec + k * (long long)p.maxlen;
    const float *a = p.a ? p.a + start : nullptr;
    const float *b = p.b + start, *f = p.f + start;
    const float *al = p.al ? p.al + start : nullptr;
    const float *w = p.w ? p.w + (p.w_stride > 0 ? k * p.w_stride : start) : nullptr;
    PqRing s{0.f, 0.f, 0.f, 0.f, sl, 0, 0.f};  // the message in ring order from lane 0
    bool ovf = false;
    const int nblocks = (cmax + 15) / 16;
    const int cnt_lo = min(mid, n - 1 - mid);  // the shorter half's update steps
    float av = 1.f, bv = 0.f, alv = 0.f, fv = 0.f, wv = 0.f;
    if (nblocks > 0) pq_half_load<U>(p, a, b, al, f, w, 0, sl, seg, n, cnt, av, bv, alv, fv, wv);
    for (int blk = 0; blk < nblocks && !ovf; ++blk) {
        float av2 = 1.f, bv2 = 0.f, alv2 = 0.f, fv2 = 0.f, wv2 = 0.f;
        if (blk + 1 < nblocks)
            pq_half_load<U>(p, a, b, al, f, w, blk + 1, sl, seg, n, cnt, av2, bv2, alv2, fv2, wv2);
        const int base = blk * 16;
        if (base + 16 <= cnt_lo)
            pq_half_steps<true, U>(s, ovf, rec, base, 16, cnt, n, seg, sl, seg_shift, av, bv, alv,
                                   fv, wv, p.alpha, p.lam);
        else
            pq_half_steps<false, U>(s, ovf, rec, base, min(16, cmax - base), cnt, n, seg, sl,
                                    seg_shift, av, bv, alv, fv, wv, p.alpha, p.lam);
        ovf = __any_sync(FULL, ovf);
        av = av2;
        bv = bv2;
        alv = alv2;
        fv = fv2;
        wv = wv2;
    }
    if (ovf) {
        // a half outgrew 16 breakpoints: the whole chain by the warp from node 0
        pq_solve_warp(p, k, start, n, lane, hdr);
        return;
    }
    PqMsg &mine = msg[warp][seg];
    if (s.idx < s.size) {  // back to ascending order from entry 0
        mine.lam[s.idx] = s.lam;
        mine.L[s.idx] = s.L;
        mine.R[s.idx] = s.R;
        mine.S[s.idx] = s.S;
    }
    if (sl == 0) {
        mine.size = cnt > 0 ? s.size : 0;
        mine.ovf = 0;
    }
    __syncwarp();
    const float am = a ? a[mid] : 1.f, alm = al ? al[mid] : p.alpha;
    const float xm = pq_root(msg[warp][0], msg[warp][1], am, b[mid], alm, f[mid], lane);
    if (lane == 0) p.x[start + mid] = xm;
    // backward over each half, outwards from the root, in processing order
    float x_next = xm;
    for (int blk = nblocks - 1; blk >= 0; --blk) {
        const int j = blk * 16 + sl;
        const bool inb = j < cnt;
        float lo = -INFINITY, hi = INFINITY;
        if (inb) {
            const float2 r = rec[node_of(j)];
            lo = r.x;
            hi = r.y;
        }
        const float xv = clip_suffix16(lo, hi, x_next, sl, inb);
        if (inb) p.x[start + node_of(j)] = xv;
        x_next = __shfl_sync(FULL, xv, 0, 16);
    }
}

// chains of 64 nodes or more: rooted at the middle node, the halves on two 16-lane
// segments of one warp; shorter ones one warp per chain from one end
void launch_pq(const PqArgs &p, long long nchains, long long max_len, WsHeader *hdr,
               cudaStream_t s)
{
    if (max_len >= 64) {
        const long long blocks = (nchains + kPqWarps - 1) / kPqWarps;
        if (!p.a && !p.al && !p.w)
            launch_k(pq_halves_kernel<true>, dim3((unsigned)blocks), dim3(kPqWarps * WARP), 0, s, p,
                     hdr);
        else
            launch_k(pq_halves_kernel<false>, dim3((unsigned)blocks), dim3(kPqWarps * WARP), 0, s,
                     p, hdr);
    } else {
        const long long blocks = (nchains + kPqWarps - 1) / kPqWarps;
        launch_k(pq_chain_kernel, dim3((unsigned)blocks), dim3(kPqWarps * WARP), 0, s, p, hdr);
    }
}

struct PqWs {
    WsHeader *hdr;
    float2 *rec;
    PqEntry *ent;
    size_t bytes;
};

PqWs carve_pq(void *base, long long nchains, long long maxlen)
{
    Carver cv(base);
    PqWs o;
    o.hdr = cv.take<WsHeader>(1);
    o.rec = cv.take<float2>((size_t)(nchains * maxlen));
    o.ent = cv.take<PqEntry>((size_t)(nchains * 2 * (3 * maxlen + 4)));
    o.bytes = align_up(cv.used, 256);
    return o;
}

// ------------------------------------------------------------- TV-l1 in 2D --
// min_x TV_h(x) + TV_v(x) + ||x - f||_1 as min_x max_y <x, y> + TV_h(x) + ||x - f||_1 -
// TV_v^*(y) (Sec. 6), by the primal-dual iteration of eq. pd at constant steps
// (tau sigma = 1, theta = 1): the dual step is the column chains of eq. prox-tv-conj,
// the primal step the row chains with piecewise-quadratic unaries of eq. prox-pq
// (scaled by tau: a = 1, b = x - tau y, alpha = tau, weights tau w_h).

// Column (dual) phase, one warp per column: c = y / sigma + xbar, weights w_v / sigma,
// y <- sigma (c - xhat).
template <bool HAS_W>
struct L1ColsP {
    static constexpr bool CREC = true;
    static constexpr bool UNIFORM_W = !HAS_W;  // one weight (a scaled lambda) per chain
    struct Raw {
        float xb, y, w;
    };
    struct Acc {};
    const float *xbar, *wv;
    float *y;
    float lam;
    long long H, W;
    float sigma, inv_sigma;

    __device__ bool resolve() { return true; }
    __device__ long long num_chains() const { return W; }
    __device__ int max_len() const { return (int)H; }
    __device__ bool chain(long long k, long long &start, int &n) const
    {
        start = k;
        n = (int)H;
        return true;
    }
    __device__ void fetch(long long col, long long, int n, int i, Raw &r) const
    {
        const bool in = i < n;
        const long long o = (long long)i * W + col;
        r.xb = in ? xbar[o] : 0.f;
        r.y = in ? y[o] : 0.f;
        r.w = HAS_W ? ((i < n - 1) ? wv[o] : 0.f) : lam;
    }
    __device__ void unary(long long, long long, int, int, const Raw &r, float &c, float &w,
                          Acc &) const
    {
        c = r.y * inv_sigma + r.xb;
        w = r.w * inv_sigma;
    }
    __device__ void unary_direct(int i, int n, long long col, long long, float &c, float &w) const
    {
        (void)c;  // from the forward-pass record
        const float wvv = (HAS_W && i < n - 1) ? wv[(long long)i * W + col] : lam;
        w = (i < n - 1) ? wvv * inv_sigma : 0.f;
    }
    __device__ void emit(long long col, long long, int i, float xhat, float c) const
    {
        y[(long long)i * W + col] = sigma * (c - xhat);
    }
    __device__ void emit_direct(int i, long long col, long long start, float xhat, float c) const
    {
        emit(col, start, i, xhat, c);
    }
    __device__ long long spill_off(long long col, long long) const { return col * (2 * H + 2); }
    __device__ void acc_init(Acc &) const {}
    __device__ void finish(Acc &, int) const {}
    __device__ void finish_empty() const {}
};

__global__ void l1_xi(long long N, const float *x, const float *y, float tau, float *xi)
{
    pdl_enter();
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < N;
         q += (long long)gridDim.x * blockDim.x)
        xi[q] = x[q] - tau * y[q];
}

// xbar = 2 x_new - x; x = x_new
__global__ void l1_relax(long long N, const float *xn, float *x, float *xbar)
{
    pdl_enter();
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < N;
         q += (long long)gridDim.x * blockDim.x) {
        const float v = xn[q];
        xbar[q] = v + (v - x[q]);
        x[q] = v;
    }
}

constexpr int kL1Threads = 256;

// TV(x) + ||x - f||_1: FP32 over at most 32 pixels per thread, FP64 beyond; the last
// block sums the block partials in a fixed order into *energy.
__global__ void __launch_bounds__(kL1Threads)
    l1_energy_kernel(const float *f, const float *wh, const float *wv, float lam, long long H,
                     long long W, const float *x, double *partials, unsigned *ticket,
                     double *energy)
{
    __shared__ double red[kL1Threads];
    __shared__ bool last;
    pdl_enter();
    const long long N = H * W;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long dr = stride / W, dc = stride - dr * W;
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long r = q / W, c = q - r * W;
    double acc = 0.0;
    float part = 0.f;
    int cnt = 0;
    for (; q < N; q += stride) {
        const float xv = x[q];
        float t = fabsf(xv - f[q]);
        if (c + 1 < W) t += (wh ? wh[r * (W - 1) + c] : lam) * fabsf(x[q + 1] - xv);
        if (r + 1 < H) t += (wv ? wv[q] : lam) * fabsf(x[q + W] - xv);
        part += t;
        if (++cnt == 32) {
            acc += (double)part;
            part = 0.f;
            cnt = 0;
        }
        c += dc;
        r += dr;
        if (c >= W) {
            c -= W;
            ++r;
        }
    }
    acc += (double)part;
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = kL1Threads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double b = 0.0;
    for (unsigned bq = threadIdx.x; bq < gridDim.x; bq += blockDim.x) b += __ldcg(partials + bq);
    red[threadIdx.x] = b;
    __syncthreads();
    for (int h = kL1Threads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *energy = red[0];
        *ticket = 0;
    }
}

struct L1Ws {
    WsHeader *hdr;
    double *energy, *partials;
    unsigned *ticket;
    float *xbar, *y, *xi, *xn, *crec;
    float2 *rec, *spill;
    PqWs pq;
    size_t bytes;
};

int l1_blocks(long long N)
{
    long long b = (N + kL1Threads * 8 - 1) / (kL1Threads * 8);
    const long long cap = 4LL * sm_count_current();
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

L1Ws carve_l1(void *base, long long H, long long W)
{
    Carver cv(base);
    L1Ws o;
    const long long N = H * W;
    o.hdr = cv.take<WsHeader>(1);
    o.energy = cv.take<double>(1);
    o.ticket = cv.take<unsigned>(1);
    o.partials = cv.take<double>((size_t)l1_blocks(N));
    o.xbar = cv.take<float>((size_t)N);
    o.y = cv.take<float>((size_t)N);
    o.xi = cv.take<float>((size_t)N);
    o.xn = cv.take<float>((size_t)N);
    o.crec = cv.take<float>((size_t)N);
    o.rec = cv.take<float2>((size_t)N);
    o.spill = cv.take<float2>((size_t)(W * (2 * H + 2)));
    char *pq_base = cv.take<char>(carve_pq(nullptr, H, W).bytes);
    o.pq = carve_pq(base ? pq_base : nullptr, H, W);
    o.bytes = align_up(cv.used, 256);
    return o;
}

int ew_blocks_pq(long long n) { return (int)std::min<long long>((n + 255) / 256, 8LL * sm_count_current()); }

}  // namespace

extern "C" {

size_t tv_chain_pq_workspace_size(int64_t num_chains, int64_t max_len)
{
    if (num_chains < 0 || max_len < 0) return 0;
    return carve_pq(nullptr, num_chains, max_len).bytes;
}

tv_status tv_chain_solve_pq(const float *d_a, const float *d_b, const float *d_alpha, float alpha,
                            const float *d_f, const float *d_w, float lambda,
                            const int64_t *d_offsets, int64_t num_chains, int64_t max_len,
                            float *d_x, void *d_workspace, size_t workspace_bytes,
                            tv_stream_t stream)
{
    clear_error();
    if (num_chains < 0 || max_len < 0 || max_len > (1LL << 28)) {
        set_error("tv_chain_solve_pq: num_chains and max_len must be >= 0 (max_len <= 2^28)");
        return TV_ERR_INVALID;
    }
    if (num_chains == 0) return TV_OK;
    if (!d_b || !d_f || !d_x || !d_workspace) {
        set_error("tv_chain_solve_pq: b, f, x and workspace must not be NULL");
        return TV_ERR_INVALID;
    }
    if ((!d_alpha && !(alpha >= 0.f && alpha < INFINITY)) ||
        (!d_w && !(lambda >= 0.f && lambda < INFINITY))) {
        set_error("tv_chain_solve_pq: alpha and lambda must be finite and >= 0");
        return TV_ERR_INVALID;
    }
    const void *ins[5] = {d_a, d_b, d_alpha, d_f, d_w};
    for (const void *q : ins)
        if (q && q == d_x) {
            set_error("tv_chain_solve_pq: x must not alias the inputs");
            return TV_ERR_INVALID;
        }
    PqWs ws = carve_pq(d_workspace, num_chains, max_len);
    if (workspace_bytes < ws.bytes) {
        set_error("tv_chain_solve_pq: workspace of %zu bytes, %zu needed", workspace_bytes, ws.bytes);
        return TV_ERR_NOMEM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    tv_status st = check_cuda(cudaMemsetAsync(ws.hdr, 0, sizeof(WsHeader), s), "memset header");
    if (st != TV_OK) return st;
    PqArgs p{d_a, d_b, d_alpha, d_f, d_w, alpha, lambda, 1.f, 0, d_offsets, num_chains,
             (int)max_len, d_x, ws.rec, ws.ent};
    const bool prof = prof_on();
    if (prof) prof_mark(PK_CHAIN, s, true);
    launch_pq(p, num_chains, max_len, ws.hdr, s);
    st = check_cuda(cudaGetLastError(), "piecewise-quadratic chain launch");
    if (st == TV_OK) note_launch();
    if (prof) prof_mark(PK_CHAIN, s, false);
    return st;
}

}  // extern "C"

extern "C" {

size_t tv2d_l1_workspace_size(int64_t H, int64_t W)
{
    if (H < 1 || W < 1) return 0;
    return carve_l1(nullptr, H, W).bytes;
}

tv_status tv2d_denoise_l1(const float *d_img, int64_t H, int64_t W, const float *d_wh,
                          const float *d_wv, float lambda, float tau, int max_iters, double tol,
                          int check_every, float *d_x, int *iters_out, double *energy_out,
                          void *d_workspace, size_t workspace_bytes, tv_stream_t stream)
{
    clear_error();
    if (H < 1 || W < 1 || H > (1LL << 28) || W > (1LL << 28) || max_iters < 1 ||
        check_every < 1 || !(tau > 0.f && tau < INFINITY)) {
        set_error("tv2d_denoise_l1: need H, W >= 1, max_iters >= 1, check_every >= 1 and a "
                  "finite tau > 0");
        return TV_ERR_INVALID;
    }
    if (!d_img || !d_x || !d_workspace) {
        set_error("tv2d_denoise_l1: img, x and workspace must not be NULL");
        return TV_ERR_INVALID;
    }
    if (!(tol >= 0.0 && tol < INFINITY) ||
        ((!d_wh || !d_wv) && !(lambda >= 0.f && lambda < INFINITY))) {
        set_error("tv2d_denoise_l1: tol and lambda must be finite and >= 0");
        return TV_ERR_INVALID;
    }
    const long long N = H * W;
    const size_t npx = (size_t)N * sizeof(float);
    {
        const char *a = (const char *)d_x, *b = (const char *)d_img;
        if (a < b + npx && b < a + npx) {
            set_error("tv2d_denoise_l1: x must not overlap the image");
            return TV_ERR_INVALID;
        }
    }
    L1Ws ws = carve_l1(d_workspace, H, W);
    if (workspace_bytes < ws.bytes) {
        set_error("tv2d_denoise_l1: workspace of %zu bytes, %zu needed", workspace_bytes, ws.bytes);
        return TV_ERR_NOMEM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    tv_status st;
    if ((st = check_cuda(cudaMemsetAsync(ws.hdr, 0, sizeof(WsHeader), s), "memset")) != TV_OK ||
        (st = check_cuda(cudaMemsetAsync(ws.pq.hdr, 0, sizeof(WsHeader), s), "memset")) != TV_OK ||
        (st = check_cuda(cudaMemsetAsync(ws.ticket, 0, sizeof(unsigned), s), "memset")) != TV_OK ||
        (st = check_cuda(cudaMemcpyAsync(d_x, d_img, npx, cudaMemcpyDeviceToDevice, s), "copy")) !=
            TV_OK ||
        (st = check_cuda(cudaMemcpyAsync(ws.xbar, d_img, npx, cudaMemcpyDeviceToDevice, s), "copy")) !=
            TV_OK ||
        (st = check_cuda(cudaMemsetAsync(ws.y, 0, npx, s), "memset")) != TV_OK)
        return st;
    const float sigma = 1.f / tau;
    const int eb = l1_blocks(N);
    double e_prev = NAN, e = NAN;
    int k = 0;
    bool done = false;
    PdlScope pdl(true);  // each kernel may become resident while its predecessor finishes
    while (k < max_iters) {
        // dual step: column chains
        if (d_wv) {
            L1ColsP<true> p{ws.xbar, d_wv, ws.y, lambda, H, W, sigma, 1.f / sigma};
            st = launch_coop(p, W, (int)H, ws.rec, ws.crec, ws.spill, ws.hdr, s, PK_COL);
        } else {
            L1ColsP<false> p{ws.xbar, d_wv, ws.y, lambda, H, W, sigma, 1.f / sigma};
            st = launch_coop(p, W, (int)H, ws.rec, ws.crec, ws.spill, ws.hdr, s, PK_COL);
        }
        if (st != TV_OK) return st;
        if ((st = check_cuda(launch_k(l1_xi, dim3(ew_blocks_pq(N)), dim3(256), 0, s, N,
                                      (const float *)d_x, (const float *)ws.y, tau, ws.xi),
                             "xi")) != TV_OK)
            return st;
        note_launch();
        // primal step: row chains with piecewise-quadratic unaries (scaled by tau)
        PqArgs p{nullptr, ws.xi, nullptr, d_img, d_wh, tau, tau * lambda, tau,
                 d_wh ? (long long)(W - 1) : 0, nullptr, H, (int)W, ws.xn, ws.pq.rec, ws.pq.ent};
        const bool prof = prof_on();
        if (prof) prof_mark(PK_ROW, s, true);
        launch_pq(p, H, W, ws.pq.hdr, s);
        if ((st = check_cuda(cudaGetLastError(), "row chains")) != TV_OK) return st;
        note_launch();
        if (prof) prof_mark(PK_ROW, s, false);
        if ((st = check_cuda(launch_k(l1_relax, dim3(ew_blocks_pq(N)), dim3(256), 0, s, N,
                                      (const float *)ws.xn, d_x, ws.xbar),
                             "relax")) != TV_OK)
            return st;
        note_launch();
        ++k;
        if (k % check_every == 0 || k == max_iters) {
            if ((st = check_cuda(launch_k(l1_energy_kernel, dim3(eb), dim3(kL1Threads), 0, s, d_img,
                                          d_wh, d_wv, lambda, H, W, (const float *)d_x, ws.partials,
                                          ws.ticket, ws.energy),
                                 "energy")) != TV_OK)
                return st;
            note_launch();
            st = check_cuda(cudaMemcpyAsync(&e, ws.energy, sizeof(double), cudaMemcpyDeviceToHost, s),
                            "read energy");
            if (st == TV_OK) st = check_cuda(cudaStreamSynchronize(s), "synchronize");
            if (st != TV_OK) return st;
            if (tol > 0.0 && e_prev == e_prev && fabs(e_prev - e) <= tol * fabs(e)) {
                done = true;
                break;
            }
            e_prev = e;
        }
    }
    if (iters_out) *iters_out = k;
    if (energy_out) *energy_out = e;
    return (done || tol == 0.0) ? TV_OK : TV_ERR_NOT_CONVERGED;
}

}  // extern "C"
