// Batched row chains, one thread per chain half, with a message update of fixed shape.
//
// The update of Sec. 4.1 removes breakpoints from both ends of the message by scans whose
// length depends on the data. Run by 32 lanes in step, every node costs the warp the
// longest scan among its lanes. Here each lane instead runs its own node sequence at its
// own pace: one iteration of the warp's loop is one fixed-shape, branch-free attempt at a
// node by every lane,
//   - load the two entries after the first breakpoint and the two before the last one,
//     compute the message values there (the forward recursion from the first breakpoint,
//     the backward one from the last, Sec. 4.1), and decide which of the first three and
//     the last three breakpoints fall below -w_i or above +w_i;
//   - if neither side removes three or more, finish the node: place lambda^- and lambda^+
//     on the segments found (Sec. 4.1, transformations (a) and (b)), push them, write the
//     records (lambda^-_i, lambda^+_i) and go on to the next node;
//   - otherwise remove two breakpoints from that side and retry the same node.
// The state is updated by selects and the three stores are predicated, so the lanes of a
// warp never take different paths through the loop body. The two sides are evaluated
// independently: a breakpoint removed on the left has a value below -w_i <= w_i and is
// never removed on the right; when the right side reaches the breakpoints removed on the
// left, lambda^+ lies on the segment starting at lambda^-. Where a probe reaches the far
// end of the message, the far end's exact value is used.
//
// Per lane the message is a linear array of S slots in shared memory (slot s of lane l at
// row s + G, column l, 8 bytes: breakpoint lambda and stored slope s_p; the true slope is
// s_p + abar), with G guard rows at each end for the probes. When a push would leave the
// array the message is moved back to its middle (a warp vote keeps that rare copy off the
// common path). A message longer than S - 4 entries sends the chain to the whole-chain
// path of the workspace.
//
// Inputs are staged by the whole warp: between rounds of T iterations the lanes' next steps
// are copied into a per-lane ring of IR slots, up to IR - T steps ahead of the slowest lane;
// a lane that reaches the end of the staged range waits for the next round. In general the
// copies are 4-byte ones into [slot][lane] (the lanes' reads never share a bank); for
// uniform chains whose length is a multiple of 4 (VEC) each lane copies 4 steps of its half
// with one 16-byte copy into [slot / 4][lane][4]. Every lane reads a different chain, so a
// copy instruction touches 32 sectors either way, and the 16-byte form needs a quarter of
// the instructions and of the L1 wavefronts per node (a right half's 4 steps lie in memory
// in reverse, read back with the element index flipped). Per-edge weights go the same way:
// a right half's step s takes edge n-2-s, which sits where step s+1's node does, so its
// lanes read the weight one staged step further on (and run a step behind the staged
// range).
//
// Algorithm 2 roots chain k at node mid = n/2: lane l < 16 runs nodes 0..mid-1, lane l + 16
// nodes n-1..mid+1; then the left lane solves the root from both messages (flat_root) and
// both lanes clip their halves outwards, in step, from the records.
#pragma once
#include "tv_halves.cuh"

namespace tvk {

constexpr int FL_S = 32;   // message slots per lane
constexpr int FL_G = 2;    // guard rows at each end
constexpr int FL_IR = 32;  // staged steps per lane
constexpr int FL_T = 8;    // loop iterations between copy rounds

template <int NIN>
struct alignas(16) FlatSmem {
    union {
        struct {
            float2 msg[FL_S + 2 * FL_G][WARP];
            float in[NIN][FL_IR][WARP];
        } f;
        struct {
            float2 rec[2][CH][WARP];
            float out[WARP * RP];
        } b;
    } u;
};

__device__ __forceinline__ float2 lds2(unsigned a)
{
    float2 e;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(e.x), "=f"(e.y) : "r"(a));
    return e;
}
__device__ __forceinline__ float lds1(unsigned a)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts2_if(bool p, unsigned a, float x, float y)
{
    asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %3, 0;\n @q st.shared.v2.f32 [%0], {%1, %2};\n}\n" ::"r"(a),
                 "f"(x), "f"(y), "r"((unsigned)p)
                 : "memory");
}
__device__ __forceinline__ void stg2_if(bool p, float2 *g, float x, float y)
{
    asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %3, 0;\n @q st.global.v2.f32 [%0], {%1, %2};\n}\n" ::"l"(g),
                 "f"(x), "f"(y), "r"((unsigned)p)
                 : "memory");
}
__device__ __forceinline__ void sts2(unsigned a, float x, float y)
{
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(x), "f"(y) : "memory");
}

// Root of h(z) = z - c + m_L(z) + m_R(z) (Algorithm 2 rooted at the middle node): each half's
// message is -w left of its first breakpoint and +w right of its last, with slope s_p + a
// right of breakpoint p (a = the half's node count); h has slope 1 left of all breakpoints.
// The two breakpoint sequences (rows FL..BL of the array at baseL, FR..BR at baseR; an empty
// half has B < F and w = 0) are walked in increasing order, h is accumulated segment by
// segment, and the root is placed on the segment where h reaches 0.
__device__ __forceinline__ float flat_root(unsigned baseL, int FL, int BL, float aL, float wL,
                                           unsigned baseR, int FR, int BR, float aR, float wR,
                                           float c)
{
    auto lam = [](unsigned base, int r) { return lds2(base + ((unsigned)r << 8)); };
    int iL = FL, iR = FR;
    float zL = iL <= BL ? lam(baseL, iL).x : INFINITY;
    float zR = iR <= BR ? lam(baseR, iR).x : INFINITY;
    float z = fminf(zL, zR);
    if (!(z < INFINITY)) return c;  // no message: z = c
    float h = z - c - (BL >= FL ? wL : 0.f) - (BR >= FR ? wR : 0.f);
    float gL = 0.f, gR = 0.f;  // slope of each message right of the breakpoints passed
    const int steps = (BL - FL + 1 > 0 ? BL - FL + 1 : 0) + (BR - FR + 1 > 0 ? BR - FR + 1 : 0);
    for (int it = 0; it <= steps; ++it) {
        const float sl = 1.f + gL + gR;
        if (h >= 0.f) return z - h / sl;
        if (iL <= BL && zL == z) {
            gL = lam(baseL, iL).y + aL;
            ++iL;
            zL = iL <= BL ? lam(baseL, iL).x : INFINITY;
        }
        if (iR <= BR && zR == z) {
            gR = lam(baseR, iR).y + aR;
            ++iR;
            zR = iR <= BR ? lam(baseR, iR).x : INFINITY;
        }
        const float s2 = 1.f + gL + gR;
        const float zn = fminf(zL, zR);
        if (!(zn < INFINITY)) return z - h / s2;
        h = fmaf(s2, zn - z, h);
        z = zn;
    }
    return z - h / (1.f + gL + gR);
}

// P: a row policy of tv_chain.cu (contiguous chains, CSR or uniform) with fields y, w, lam
// and chain(); HAS_W = per-edge weights w. VEC: 16-byte staging (uniform chains, length a
// multiple of 4, y and w 16-byte aligned).
template <class P, bool VEC>
__global__ void chain_flat_kernel(P p_in, float2 *rec, float2 *spill, WsHeader *hdr, int halfmax)
{
    constexpr bool HAS_W = P::WI >= 0;
    constexpr int NIN = HAS_W ? 2 : 1;
    constexpr int S = FL_S, G = FL_G, IR = FL_IR, T = FL_T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    P p = p_in;
    if (!p.resolve()) return;
    const int lane = threadIdx.x & (WARP - 1);
    const int warp = threadIdx.x / WARP;
    const int wpb = blockDim.x / WARP;
    FlatSmem<NIN> *sm = reinterpret_cast<FlatSmem<NIN> *>(smem_raw) + warp;
    const long long wg = (long long)blockIdx.x * wpb + warp;
    const long long wc0 = wg * HW;
    const long long k = wc0 + (lane & (HW - 1));
    const bool left = lane < HW;
    long long start = 0;
    int n = 0;
    if (k < p.num_chains()) {
        if (!p.chain(k, start, n)) {
            if (left) atomicOr(&hdr->status, ERR_BAD_CHAIN);
            n = 0;
        }
    }
    const int mid = n >> 1;
    const int cnt = n == 0 ? 0 : (left ? mid : n - 1 - mid);  // steps of this half
    const int cmax = __reduce_max_sync(FULL, cnt);
    float2 *rec_w = rec + wg * (long long)halfmax * WARP;

    // ---------------- staging: step t of this half at in[a][t % IR][lane] ----------------
    // left: node t (weight of edge t -> t+1); right: node n-1-t (weight of edge n-2-t -> n-1-t)
    const float *ysrc = p.y + start + (left ? 0 : n - 1);
    const float *wsrc = nullptr;
    if constexpr (HAS_W) wsrc = p.w + start + (left ? 0 : n - 2);
    const long long dir = left ? 1 : -1;
    // VEC: steps 4q..4q+3 at in[a][4 (q % (IR/4)) ...] as [slot/4][lane][4]; a right half's
    // chunk is nodes n-4-4q..n-1-4q in memory order (step 4q+e at element 3-e). A right
    // half's weights are read one step further on (edge n-2-s at step s+1's place), so its
    // chunks run to step cnt: nodes from mid-3 >= 0 (n = 4: the chunk of step 0 only).
    float *const in4 = &sm->u.f.in[0][0][0] + 4 * lane;
    const int wlag = VEC && HAS_W && !left ? 1 : 0;
    const int cnt_st = cnt > 0 ? cnt + wlag : 0;  // staged steps (none for an empty half)
    auto stage = [&](int t0, int t1) {  // steps [t0, t1), warp-uniform bounds
        if constexpr (VEC) {
            for (int t = t0; t < t1; t += 4)
                if (t < cnt_st) {
                    const int o = ((t >> 2) & (IR / 4 - 1)) * (4 * WARP);
                    cp_async16(in4 + o, left ? ysrc + t : ysrc - t - 3);
                    if constexpr (HAS_W)
                        cp_async16(in4 + IR * WARP + o, left ? wsrc + t : wsrc - t - 2);
                }
        } else {
            for (int t = t0; t < t1; ++t) {
                if (t < cnt) {
                    cp_async4(&sm->u.f.in[0][t & (IR - 1)][lane], ysrc + dir * t);
                    if constexpr (HAS_W)
                        cp_async4(&sm->u.f.in[NIN - 1][t & (IR - 1)][lane], wsrc + dir * t);
                }
            }
        }
        cp_async_commit();
    };
    // staged ranges end on 4-step boundaries for VEC (the chunk past a half's end stays in
    // its chain: node mid + 2 at most on the left, mid - 2 at least on the right)
    const int cmaxs = VEC ? (cmax + (HAS_W ? 4 : 3)) & ~3 : cmax;
    auto stage_end = [&](int t) { return VEC ? t & ~3 : t; };

    // ---------------- message array ----------------
    const unsigned msg0 = (unsigned)__cvta_generic_to_shared(&sm->u.f.msg[0][lane]);
    auto slot = [&](int s) { return msg0 + ((unsigned)(s + G) << 8); };
    const unsigned lo_lim = slot(1), hi_lim = slot(S - 2);
    const unsigned in0 = VEC ? (unsigned)__cvta_generic_to_shared(in4)
                             : (unsigned)__cvta_generic_to_shared(&sm->u.f.in[0][0][lane]);
    const unsigned flip = VEC && !left ? 3u : 0u;
    auto in_addr = [&](int t) {
        return VEC ? in0 + (((unsigned)(t >> 2) & (IR / 4 - 1)) << 9) + ((((unsigned)t & 3u) ^ flip) << 2)
                   : in0 + ((unsigned)(t & (IR - 1)) << 7);
    };

    int hi = 0;      // steps < hi are staged and their copies complete
    int issued = 0;  // steps < issued have copies issued
    {
        const int t1 = min(cmaxs, IR - T);
        stage(0, t1);
        issued = t1;
        cp_async_wait<0>();
        hi = issued;
    }

    unsigned PF = slot(S / 2 - 1), PB = slot(S / 2);  // shared addresses of the first and last breakpoint
    float fl = 0.f, fs = 0.f, bl = 0.f;  // first breakpoint (lambda, stored slope), last lambda
    float uF = 0.f, uB = 0.f;         // message values at the first / last breakpoint
    float ab = 1.f, wprev = 0.f;
    bool fresh = true;                // the current node has not been started
    bool alive = true;
    int j = 0;
    bool fw = cnt > 0;
    if (fw) {  // leaf node: m^(z) = z - c has slope 1, lambda^-+ = c -+ w
        const float c = lds1(in_addr(0));
        const float w0 = HAS_W ? lds1(in_addr(wlag) + IR * 128) : p.lam;
        PF = slot(S / 2 - 1);
        PB = PF + 256;
        fl = c - w0;
        fs = 0.f;
        bl = c + w0;
        sts2(PF, fl, 0.f);
        sts2(PB, bl, -1.f);
        rec_w[lane] = make_float2(fl, bl);
        wprev = w0;
        ab = 2.f;
        j = 1;
        fw = j < cnt;
    }

    // ---------------- forward pass, each lane at its own pace ----------------
    // Rounds of T loop iterations; between rounds the warp refills the staging rings. In an
    // iteration a lane with a staged node either finishes it or removes two breakpoints.
    for (;;) {
        __syncwarp();
        const int jmin = __reduce_min_sync(FULL, fw ? j : 0x7fffffff);
        if (jmin == 0x7fffffff) break;
        cp_async_wait<0>();
        hi = issued;
        {
            const int t1 = min(cmaxs, stage_end(jmin + IR - T));
            if (t1 > issued) {
                stage(issued, t1);
                issued = t1;
            }
        }
#pragma unroll 1
        for (int it = 0; it < T; ++it) {
            const bool act = fw && j + wlag < hi;
            const unsigned ia = in_addr(j);
            const float c = lds1(ia);
            const float w = HAS_W ? lds1((VEC ? in_addr(j + wlag) : ia) + IR * 128) : p.lam;
            const float nw = -w;
            const float uF0 = fresh ? fl - c - wprev : uF;
            const float uB0 = fresh ? bl - c + wprev : uB;
            const unsigned d = PB - PF;  // (entries - 1) * 256
            const bool m2 = d >= 256u, m3 = d >= 512u, d2 = d == 256u, d3 = d == 512u;
            const float2 e1 = lds2(PF + 256), e2 = lds2(PF + 512);
            const float2 g1 = lds2(PB - 256), g2 = lds2(PB - 512);
            const float sl1 = fs + ab, sl2 = e1.y + ab;
            const float r1 = g1.y + ab, r2 = g2.y + ab;
            float u1 = fmaf(sl1, e1.x - fl, uF0);
            float u2 = fmaf(sl2, e2.x - e1.x, u1);
            float v1 = fmaf(-r1, bl - g1.x, uB0);
            float v2 = fmaf(-r2, g1.x - g2.x, v1);
            u1 = d2 ? uB0 : u1;
            v1 = d2 ? uF0 : v1;
            u2 = d3 ? uB0 : u2;
            v2 = d3 ? uF0 : v2;
            const bool p0 = uF0 < nw, p1 = p0 && m2 && u1 < nw, p2 = p1 && m3 && u2 < nw;
            const bool q0 = uB0 > w, q1 = q0 && m2 && v1 > w, q2 = q1 && m3 && v2 > w;
            // lambda^- / lambda^+ as if the node finishes now
            const float al = p1 ? e1.x : fl;
            const float av = p1 ? u1 : uF0;
            const float asl = p1 ? sl2 : (p0 ? sl1 : 1.f);
            const float as = p1 ? e1.y : (p0 ? fs : 1.f - ab);
            const float lm = al + slope_div(nw - av, asl);
            const unsigned nPF = p1 ? PF + 256 : (p0 ? PF : PF - 256);
            const unsigned kPB = q1 ? PB - 512 : (q0 ? PB - 256 : PB);
            const bool flm = kPB <= nPF;
            const float ar = flm ? lm : (q1 ? g1.x : bl);
            const float avr = flm ? nw : (q1 ? v1 : uB0);
            const float asr = flm ? as + ab : (q1 ? r2 : (q0 ? r1 : 1.f));
            const float hp = ar + slope_div(w - avr, asr);
            const unsigned nPB = (flm ? nPF : kPB) + 256;
            const bool done = act && !p2 && !q2;  // the node finishes
            const bool cL = act && p2;            // remove two on the left and retry
            const bool cR = act && !p2 && q2;     // remove two on the right and retry
            sts2_if(done, nPF, lm, as);
            sts2_if(done, nPB, hp, -ab);
            stg2_if(done, rec_w + (long long)j * WARP + lane, lm, hp);
            PF = done ? nPF : (cL ? PF + 512 : PF);
            PB = done ? nPB : (cR ? PB - 512 : PB);
            fl = done ? lm : (cL ? e2.x : fl);
            fs = done ? as : (cL ? e2.y : fs);
            bl = done ? hp : (cR ? g2.x : bl);
            uF = cL ? (d3 ? uB0 : u2) : uF0;
            uB = cR ? (d3 ? uF0 : v2) : uB0;
            fresh = done || (fresh && !act);
            wprev = done ? w : wprev;
            ab = done ? ab + 1.f : ab;
            j = done ? j + 1 : j;
            fw = done ? j < cnt : fw;
            const bool rc = done && (PF < lo_lim || PB > hi_lim);
            if (__any_sync(FULL, rc)) {
                if (rc) {
                    // move the message back to the middle of the array
                    const int mm = (int)((PB - PF) >> 8) + 1;
                    if (mm > S - 4) {
                        alive = false;
                        fw = false;
                    } else {
                        const unsigned dst = slot((S - mm) >> 1);
                        if (dst < PF) {
                            for (int q = 0; q < mm; ++q) {
                                const float2 e = lds2(PF + ((unsigned)q << 8));
                                sts2(dst + ((unsigned)q << 8), e.x, e.y);
                            }
                        } else {
                            for (int q = mm - 1; q >= 0; --q) {
                                const float2 e = lds2(PF + ((unsigned)q << 8));
                                sts2(dst + ((unsigned)q << 8), e.x, e.y);
                            }
                        }
                        PB = dst + (PB - PF);
                        PF = dst;
                    }
                }
            }
        }
    }
    cp_async_wait<0>();
    __syncwarp();

    // ---------------- root ----------------
    const int F = (int)((PF - msg0) >> 8), B = (int)((PB - msg0) >> 8);
    const int FR = __shfl_down_sync(FULL, F, HW), BR = __shfl_down_sync(FULL, B, HW);
    const float wR = __shfl_down_sync(FULL, wprev, HW);
    const int cntR = __shfl_down_sync(FULL, cnt, HW);
    const bool aliveR = __shfl_down_sync(FULL, (int)alive, HW) != 0;
    const bool ok = __shfl_sync(FULL, (int)(alive && aliveR), lane & (HW - 1)) != 0;
    float xroot = 0.f;
    if (left && n > 0 && ok) {
        float c_root, w_unused;
        p.unary_direct(mid, n, k, start, c_root, w_unused);
        xroot = flat_root(msg0, cnt > 0 ? F : 0, cnt > 0 ? B : -1, (float)cnt, wprev,
                          msg0 + HW * 8, cntR > 0 ? FR : 0, cntR > 0 ? BR : -1, (float)cntR, wR,
                          c_root);  // lane + 16's array is 16 columns along
        p.emit_direct(mid, k, start, xroot, c_root);
    }
    xroot = __shfl_sync(FULL, xroot, lane & (HW - 1));
    __syncwarp();

    // ---------------- backward pass, outwards from the root, in step ----------------
    const int cnt_eff = ok ? cnt : 0;
    float xv = xroot;
    const bool vout = p.out_vec();
    float *dst = p.x + start;
    auto load_recs = [&](int buf, int ch) {
#pragma unroll 4
        for (int u = 0; u < CH; ++u) {
            const int jj = ch * CH + u;
            if (jj < cnt_eff) cp_async8(&sm->u.b.rec[buf][u][lane], rec_w + (long long)jj * WARP + lane);
        }
    };
    const int nchunks = (cmax + CH - 1) / CH;
    int b = 0;
    if (nchunks > 0) load_recs(0, nchunks - 1);
    cp_async_commit();
    for (int ch = nchunks - 1; ch >= 0; --ch) {
        if (ch > 0) load_recs(b ^ 1, ch - 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncwarp();
        if (vout) {
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
                if (j0 + 3 < cnt_eff) {
                    *reinterpret_cast<float4 *>(dst + lo) = left ? make_float4(xs[0], xs[1], xs[2], xs[3])
                                                                 : make_float4(xs[3], xs[2], xs[1], xs[0]);
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (j0 + e < cnt_eff) dst[left ? lo + e : lo + 3 - e] = xs[e];
                }
            }
        } else {
#pragma unroll 4
            for (int jj = CH - 1; jj >= 0; --jj) {
                const int t = ch * CH + jj;
                if (t < cnt_eff) {
                    const float2 r = sm->u.b.rec[b][jj][lane];
                    xv = clip_to(xv, r.x, r.y);
                    dst[left ? t : n - 1 - t] = xv;
                }
            }
        }
        __syncwarp();
        b ^= 1;
    }
    cp_async_wait<0>();
    if (left && n > 0 && !ok) {
        atomicAdd(&hdr->overflowed, 1ull);
        half_fallback(p, k, start, n, spill + p.spill_off(k, start), rec_w + lane,
                      (float *)nullptr);
    }
}

}  // namespace tvk
