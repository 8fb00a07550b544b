// Device-side dynamic program for TV-l2 on a chain (Algorithm 2 specialised to
// quadratic unaries, Sec. 4.1), and the warp-level machinery that runs one chain
// per thread over a batch of chains.
//
// Normalised problem on a chain of n nodes (eq. 1D-ROF with a_i = 1, b_i = c_i):
//     x* = argmin_x sum_i 1/2 (x_i - c_i)^2 + sum_{i<n-1} w_i |x_{i+1} - x_i|
//
// The current message is a sequence of breakpoints lambda_p (increasing) with a
// stored slope s_p for the segment to the right of each breakpoint. The true
// slope at node i (0-based) is s_p + abar with abar = i + 1 (Sec. 4.1, implicit
// slopes: adding a_i = 1 to every segment costs nothing). The message value at
// the first breakpoint is -w_{i-1} and at the last one +w_{i-1}, so values are
// recomputed from the ends by the forward/backward recursions of Sec. 4.1 and
// never stored. All slopes are small integers held exactly in float32.
//
// Per thread the sequence lives in a ring of RING entries in shared memory
// (entry j of lane l at ring[(j mod RING)][l], so a lane always hits its own
// bank). A sequence that would outgrow the ring is finished later from a
// global-memory two-ended array of 2n+2 entries (the bound of Sec. 4.1).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace tvk {

// Optional policy hooks of the one-thread-per-chain kernel, for policies whose
// warps each serve one group of chains of a larger structure (the batched images):
//   bool bind_warp(warp_chain0)   per-warp set-up; false skips the whole warp
//   long long col_base(warp_chain0)   column index of lane 0 (column layouts)
//   long long rec_slot(wg, max_len)   first record of warp wg (default wg*max_len*32)
template <class P, class = void>
struct has_bind : std::false_type {};
template <class P>
struct has_bind<P, std::void_t<decltype(std::declval<P &>().bind_warp(0LL))>> : std::true_type {};
template <class P, class = void>
struct has_col_base : std::false_type {};
template <class P>
struct has_col_base<P, std::void_t<decltype(std::declval<const P &>().col_base(0LL))>>
    : std::true_type {};
template <class P, class = void>
struct has_rec_slot : std::false_type {};
template <class P>
struct has_rec_slot<P, std::void_t<decltype(std::declval<const P &>().rec_slot(0LL, 0))>>
    : std::true_type {};

template <class P>
__device__ __forceinline__ long long col_base_of(const P &p, long long warp_chain0)
{
    if constexpr (has_col_base<P>::value) return p.col_base(warp_chain0);
    else return warp_chain0;
}

constexpr int WARP = 32;
constexpr int CH = 8;   // nodes per staged chunk
constexpr int QPC = CH / 4;  // 16-byte quads per chain and chunk

// Device error word bits (workspace header).
constexpr int ERR_BAD_CHAIN = 1;
constexpr int ERR_CAPACITY = 2;  // a message outgrew its storage (chain left NaN)

struct WsHeader {
    int status;              // ERR_* bits, sticky until read
    int pad0;
    unsigned long long overflowed;  // chains finished from the global reserve
    unsigned char pad[48];
};
static_assert(sizeof(WsHeader) == 64, "header size");

struct DPState {
    int F, B;           // logical indices of the first and last breakpoint
    float fl, fs;       // entry F (lambda, stored slope)
    float bl, bs;       // entry B
    float w_prev;       // weight of the edge into the current node
};

// Message sequence of one chain in a ring of RING entries in shared memory:
// entry j of this lane at byte offset ((j mod RING) * 32 + lane) * 8 of the ring.
template <int RING>
struct RingStore {
    unsigned base;  // shared-window address of ring[0][lane]
    static constexpr int cap = RING;
    __device__ __forceinline__ unsigned addr(int j) const
    {
        return base + ((unsigned)(j & (RING - 1)) << 8);  // 32 lanes * 8 bytes per slot row
    }
    __device__ __forceinline__ float2 ld(int j) const
    {
        float2 e;
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(e.x), "=f"(e.y) : "r"(addr(j)));
        return e;
    }
    __device__ __forceinline__ void st(int j, float2 e) const
    {
        asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(addr(j)), "f"(e.x), "f"(e.y)
                     : "memory");
    }
};

struct LinearStore {
    float2 *base;  // 2n+2 entries; logical index j at base[j]
    static constexpr int cap = 0x7fffffff;
    __host__ __device__ __forceinline__ float2 ld(int j) const { return base[j]; }
    __host__ __device__ __forceinline__ void st(int j, float2 e) const { base[j] = e; }
};

// Node 0: m^_0(z) = z - c_0 has slope 1, so lambda^-_0 = c_0 - w_0, lambda^+_0 = c_0 + w_0.
// Quotient by a small positive integer slope: fast reciprocal on the device.
__host__ __device__ __forceinline__ float slope_div(float num, float slope)
{
#ifdef __CUDA_ARCH__
    return __fdividef(num, slope);
#else
    return num / slope;
#endif
}

template <class S>
__host__ __device__ __forceinline__ void dp_first(DPState &d, const S &s, int F0, float c0, float w0,
                                         float &lm, float &hp)
{
    lm = c0 - w0;
    hp = c0 + w0;
    d.F = F0;
    d.B = F0 + 1;
    d.fl = lm;
    d.fs = 0.f;   // true slope 1 between the two breakpoints
    d.bl = hp;
    d.bs = -1.f;  // -abar_0: the clipped flat right end
    d.w_prev = w0;
    s.st(d.F, make_float2(d.fl, d.fs));
    s.st(d.B, make_float2(d.bl, d.bs));
}

// Message update for node i >= 1 (abar = i + 1), transformations (a) and (b) of
// Sec. 4.1: the left scan removes breakpoints with m^_i < -w_i and places
// lambda^- on the segment to the right of the last one removed (or on the left
// end segment, slope a_i = 1, if none was removed); the right scan does the
// mirror image with +w_i over the breakpoints the left scan kept. Returns false,
// leaving the store and state untouched, if the new sequence would exceed `cap`.
//
// Each scan carries an "anchor" (lambda, value, slope of the segment on which the
// new breakpoint would lie) so that both placements are one formula,
// lambda = anchor + (+-w_i - value) / slope, whatever the number removed; a warp
// then runs one compact loop per side for as many removals as its slowest lane
// needs. Quotients by the integer slopes use the fast reciprocal (2 ulp).
template <class S>
__host__ __device__ __forceinline__ bool dp_step(DPState &d, const S &s, int cap, float ci, float wi,
                                                 float abar, float &lm, float &hp)
{
    const int F = d.F, B = d.B;
    const float nwi = -wi;

    // ---------------- left scan (forward recursion from the first breakpoint) ----
    const float vF = d.fl - ci - d.w_prev;  // m^_i(lambda_F): incoming value -w_{i-1}
    float al = d.fl, av = vF, asl = 1.f, as = 1.f - abar;  // anchor: nothing removed
    int lastL = F - 1;
    {
        int p = F;
        float pl = d.fl, ps = d.fs, v = vF;
        bool go = v < nwi;
        while (go) {  // remove breakpoint p
            al = pl;
            av = v;
            asl = ps + abar;
            as = ps;
            lastL = p;
            if (p == B) break;
            const float2 q = s.ld(p + 1);
            v = fmaf(asl, q.x - pl, v);
            ++p;
            pl = q.x;
            ps = q.y;
            go = v < nwi;
        }
    }
    // Both end values of m^_i are known exactly (-w_{i-1} + lambda_F - c_i at the
    // first breakpoint, w_{i-1} + lambda_B - c_i at the last). When the scan
    // stopped nearer the last breakpoint, re-evaluate the anchor's value by the
    // backward recursion from there: the same value in exact arithmetic, but FP32
    // rounding of the breakpoints is no longer multiplied by the large slopes of
    // the segments crossed. The walk is shorter than the scan, so the update
    // stays O(d_i + 1).
    if (lastL - F > B - lastL) {
        float vb = d.bl - ci + d.w_prev;
        float ql = d.bl;
        for (int q = B - 1; q >= lastL; --q) {
            const float2 e = s.ld(q);
            vb = fmaf(-(e.y + abar), ql - e.x, vb);
            ql = e.x;
        }
        av = vb;
    }
    lm = al + slope_div(nwi - av, asl);
    const float lm_s = as;

    // ---------------- right scan (backward recursion from the last breakpoint) ---
    // over the breakpoints with index > lastL
    float bl2 = d.bl, bv = d.bl - ci + d.w_prev, bsl = 1.f;  // anchor: nothing removed
    int lastR = B + 1;
    bool from_lm = B <= lastL;  // every breakpoint went left of lambda^-
    if (!from_lm) {
        int q = B;
        float ql = d.bl, v = bv;
        bool go = v > wi;
        while (go) {  // remove breakpoint q
            lastR = q;
            if (q - 1 <= lastL) {
                from_lm = true;  // lambda^+ on the segment that starts at lambda^-
                break;
            }
            const float2 e = s.ld(q - 1);
            const float sl = e.y + abar;
            bl2 = ql;
            bv = v;
            bsl = sl;
            v = fmaf(-sl, ql - e.x, v);
            --q;
            ql = e.x;
            go = v > wi;
        }
        // mirror image of the re-evaluation above
        if (!from_lm && lastR <= B && B - lastR > lastR - F) {
            float vf = vF;
            float el = d.fl, es = d.fs;
            for (int t = F + 1; t <= lastR; ++t) {
                const float2 e2 = s.ld(t);
                vf = fmaf(es + abar, e2.x - el, vf);
                el = e2.x;
                es = e2.y;
            }
            bv = vf;
        }
    }
    if (from_lm) {
        bl2 = lm;
        bv = nwi;
        bsl = lm_s + abar;
    }
    hp = bl2 + slope_div(wi - bv, bsl);

    const int nF = lastL;
    const int keptR = lastR - 1;  // last breakpoint kept on the right
    const int nB = (keptR > nF ? keptR : nF) + 1;
    if (nB - nF + 1 > cap) return false;
    s.st(nF, make_float2(lm, lm_s));
    s.st(nB, make_float2(hp, -abar));
    d.F = nF;
    d.B = nB;
    d.fl = lm;
    d.fs = lm_s;
    d.bl = hp;
    d.bs = -abar;
    d.w_prev = wi;
    return true;
}

// Programmatic dependent launch (griddepcontrol, sm_90 and later). A grid launched with
// a programmatic dependency on the previous kernel of its stream is launched as that
// kernel's blocks exit, before the kernel as a whole has completed; wait blocks until
// the previous grid has completed and its memory is visible. For a grid launched
// without the dependency it is a no-op. Called first thing by every kernel that may be
// launched this way. (The kernels do not release their dependents early: blocks of the
// next phase placed while this one still fills the SMs would be spread unevenly.)
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

__device__ __forceinline__ float clip_to(float v, float lo, float hi)
{
    return fminf(fmaxf(v, lo), hi);
}

// ------------------------------------------------------------------ cp.async --
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ------------------------------------------------------------ warp machinery --
//
// One warp owns 32 chains, one per lane; all lanes walk their chains node by node
// in step, so the warp stages the next CH nodes of every chain in shared memory
// with asynchronous copies while it works on the current ones.
//
// Tiles. Rows (contiguous chains): chain-major, lane l's nodes at [l*RP + j] with
// RP = CH + 4 so rows stay 16-byte aligned; a lane reads four nodes at once
// (128-bit loads by the 32 lanes hit distinct bank groups). Columns (node i of
// chain k at i*ld + k): node-major, [j*CP + l] with CP = 32 + 4, so that one
// 16-byte copy brings four neighbouring columns and every lane reads its own bank;
// slot 32 of a node row holds the first column of the next warp (horizontal
// neighbour of lane 31).
//
// A phase policy P describes one batch of chains and what surrounds the DP:
//   COLS, NIN, NEIGH (stage input 0 of the column to the right), CREC (record c_i
//   for the epilogue), NOUT (row-layout outputs); resolve(), num_chains(),
//   max_len(), chain(k, &start, &n); in_ptr(a), in_off(a, k, start) (rows),
//   in_ld(a), in_kmax(a) (cols), in_lim(a, n), in_vec(a) (16-byte copies allowed);
//   unary(v[], xr, j, i, n, k, &c, &w, acc): c_i and the weight w_i of edge
//   i -> i+1 from the staged values of node i; unary_direct(...) the same from
//   global memory (overflow path); emit_cols / emit_direct, out_ptr(o),
//   out_off(o, k, start), out_vec(); spill_off(k, start); acc_init / finish /
//   finish_empty (end-of-warp hooks, e.g. gap partials).

constexpr int RP = CH + 4;
constexpr int CP = WARP + 4;

// The forward pass uses the input tiles and the ring, the backward pass the record
// tiles and the output tile: the two sets share their shared memory.
template <class P, int RING>
struct alignas(16) WarpSmem {
    union {
        struct {
            float in[P::NIN][2][P::COLS ? CH * CP : WARP * RP];
            float2 ring[RING][WARP];
        } f;
        struct {
            float2 rec[2][CH][WARP];
            float crec[P::CREC ? 2 : 1][P::CREC ? CH : 1][WARP];
            float out[P::COLS ? 4 : WARP * RP];
        } b;
    } u;
    long long start[WARP];
    int len[WARP];
};

template <class P, int RING>
__device__ __forceinline__ void fill_inputs(const P &p, WarpSmem<P, RING> *sm, int b, int chunk,
                                            int lane, long long warp_chain0)
{
#pragma unroll
    for (int a = 0; a < P::NIN; ++a) {
        const float *src = p.in_ptr(a);
        if (src == nullptr) continue;  // an optional input this warp does not have
        float *tile = sm->u.f.in[a][b];
        if constexpr (P::COLS) {
            const long long kb = col_base_of(p, warp_chain0);
            const long long ld = p.in_ld(a);
            const long long kmax = p.in_kmax(a);
            const int lim = p.in_lim(a, p.max_len());
            if (p.in_vec(a)) {
                // 4 node rows of 32 columns per instruction, 16 bytes per lane
#pragma unroll
                for (int u = 0; u < CH / 4; ++u) {
                    const int jn = 4 * u + (lane >> 3);
                    const int i = chunk * CH + jn;
                    const int c4 = (lane & 7) * 4;
                    const long long k = kb + c4;
                    if (i < lim) {
                        if (k + 3 < kmax) {
                            cp_async16(&tile[jn * CP + c4], src + (long long)i * ld + k);
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (k + e < kmax)
                                    cp_async4(&tile[jn * CP + c4 + e], src + (long long)i * ld + k + e);
                        }
                    }
                }
            } else {
                const long long k = kb + lane;
                if (k < kmax) {
#pragma unroll 4
                    for (int u = 0; u < CH; ++u) {
                        const int i = chunk * CH + u;
                        if (i < lim) cp_async4(&tile[u * CP + lane], src + (long long)i * ld + k);
                    }
                }
            }
            if (P::NEIGH && a == 0 && lane < CH) {
                const long long kn = kb + WARP;
                const int i = chunk * CH + lane;
                if (kn < kmax && i < lim) cp_async4(&tile[lane * CP + WARP], src + (long long)i * ld + kn);
            }
        } else {
            if (p.in_vec(a)) {
                // 32 / QPC chains x CH nodes per instruction, 16 bytes per lane
#pragma unroll
                for (int u = 0; u < CH / 4; ++u) {
                    const int t = u * WARP + lane;
                    const int jj = t / QPC, q = (t % QPC) * 4;
                    const int i = chunk * CH + q;
                    if (i < p.in_lim(a, sm->len[jj]))
                        cp_async16(&tile[jj * RP + q],
                                   src + p.in_off(a, warp_chain0 + jj, sm->start[jj]) + i);
                }
            } else {
#pragma unroll 4
                for (int u = 0; u < CH; ++u) {
                    const int t = u * WARP + lane;
                    const int jj = t / CH, node = t % CH;
                    const int i = chunk * CH + node;
                    if (i < p.in_lim(a, sm->len[jj]))
                        cp_async4(&tile[jj * RP + node],
                                  src + p.in_off(a, warp_chain0 + jj, sm->start[jj]) + i);
                }
            }
        }
    }
}

template <class P, int RING>
__device__ __forceinline__ void fill_records(WarpSmem<P, RING> *sm, int b, int chunk, int lane,
                                             const float2 *rec_w, const float *crec_w, int n)
{
#pragma unroll 4
    for (int u = 0; u < CH; ++u) {
        const int i = chunk * CH + u;
        if (i < n) {
            cp_async8(&sm->u.b.rec[b][u][lane], rec_w + (long long)i * WARP + lane);
            if constexpr (P::CREC)
                cp_async4(&sm->u.b.crec[b][u][lane], crec_w + (long long)i * WARP + lane);
        }
    }
}

template <class P, int RING>
__device__ __forceinline__ void flush_outputs(const P &p, WarpSmem<P, RING> *sm, int chunk,
                                              int lane, long long warp_chain0, int o)
{
    float *dst = p.out_ptr(o);
    if (p.out_vec()) {
#pragma unroll
        for (int u = 0; u < CH / 4; ++u) {
            const int t = u * WARP + lane;
            const int jj = t / QPC, q = (t % QPC) * 4;
            const int i = chunk * CH + q;
            if (i < sm->len[jj])
                *reinterpret_cast<float4 *>(dst + p.out_off(o, warp_chain0 + jj, sm->start[jj]) + i) =
                    *reinterpret_cast<const float4 *>(&sm->u.b.out[jj * RP + q]);
        }
    } else {
#pragma unroll 4
        for (int u = 0; u < CH; ++u) {
            const int t = u * WARP + lane;
            const int jj = t / CH, node = t % CH;
            const int i = chunk * CH + node;
            if (i < sm->len[jj])
                dst[p.out_off(o, warp_chain0 + jj, sm->start[jj]) + i] = sm->u.b.out[jj * RP + node];
        }
    }
}

// Overflow path: one lane re-solves its whole chain from global memory, with the
// message in a two-ended array of 2n+2 entries started in its middle (Sec. 4.1).
template <class P>
__device__ void solve_chain_global(const P &p, long long k, long long start, int n,
                                   float2 *spill, float2 *rec_w, const float *crec_w, int lane)
{
    LinearStore S{spill};
    DPState d;
    float lm, hp, c, w;
    float xlast = 0.f;
    for (int i = 0; i < n; ++i) {
        p.unary_direct(i, n, k, start, c, w);
        if constexpr (P::CREC) c = crec_w[(long long)i * WARP + lane];  // recorded c_i
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
        else rec_w[(long long)i * WARP + lane] = make_float2(lm, hp);
    }
    float xv = xlast;
    for (int i = n - 1; i >= 0; --i) {
        float cc = 0.f;
        if constexpr (P::CREC) cc = crec_w[(long long)i * WARP + lane];
        if (i < n - 1) {
            const float2 r = rec_w[(long long)i * WARP + lane];
            xv = clip_to(xv, r.x, r.y);
        }
        p.emit_direct(i, k, start, xv, cc);
    }
}

__device__ __forceinline__ float pick4(const float4 &q, int e)
{
    return e == 0 ? q.x : (e == 1 ? q.y : (e == 2 ? q.z : q.w));
}

template <class P, int RING>
__global__ void __launch_bounds__(128) chain_batch_kernel(P p_in, float2 *rec, float *crec,
                                                          float2 *spill, WsHeader *hdr)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    P p = p_in;
    if (!p.resolve()) return;  // e.g. the 2D iteration has already converged
    const int lane = threadIdx.x & (WARP - 1);
    const int warp = threadIdx.x / WARP;
    const int wpb = blockDim.x / WARP;
    WarpSmem<P, RING> *sm = reinterpret_cast<WarpSmem<P, RING> *>(smem_raw) + warp;
    const long long wg = (long long)blockIdx.x * wpb + warp;
    const long long warp_chain0 = wg * WARP;
    const long long k = warp_chain0 + lane;
    if constexpr (has_bind<P>::value) {
        if (warp_chain0 >= p.num_chains() || !p.bind_warp(warp_chain0)) {
            p.finish_empty();
            return;
        }
    }
    const int max_len = p.max_len();

    long long start = 0;
    int n = 0;
    if (k < p.num_chains()) {
        if (!p.chain(k, start, n)) {
            atomicOr(&hdr->status, ERR_BAD_CHAIN);
            n = 0;
        }
    }
    sm->start[lane] = start;
    sm->len[lane] = n;
    int nmax = n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
    __syncwarp();
    if (nmax == 0) {
        p.finish_empty();
        return;
    }
    const int nchunks = (nmax + CH - 1) / CH;
    long long slot = wg * (long long)max_len * WARP;
    if constexpr (has_rec_slot<P>::value) slot = p.rec_slot(wg, max_len);
    float2 *rec_w = rec + slot;
    float *crec_w = P::CREC ? crec + slot : nullptr;

    RingStore<RING> S{(unsigned)__cvta_generic_to_shared(&sm->u.f.ring[0][lane])};
    DPState d;
    typename P::Acc acc;
    p.acc_init(acc);
    bool alive = true;
    float xlast = 0.f;

    // ---------------- forward pass ----------------
    fill_inputs(p, sm, 0, 0, lane, warp_chain0);
    cp_async_commit();
    int b = 0;
    for (int ch = 0; ch < nchunks; ++ch) {
        if (ch + 1 < nchunks) fill_inputs(p, sm, b ^ 1, ch + 1, lane, warp_chain0);
        cp_async_commit();
        cp_async_wait<1>();
        __syncwarp();
#pragma unroll 1
        for (int j4 = 0; j4 < CH; j4 += 4) {
            float4 q[P::NIN];
            if constexpr (!P::COLS) {
#pragma unroll
                for (int a = 0; a < P::NIN; ++a)
                    q[a] = *reinterpret_cast<const float4 *>(&sm->u.f.in[a][b][lane * RP + j4]);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = j4 + e;
                const int i = ch * CH + j;
                float v[P::NIN];
                float xr = 0.f;
                if constexpr (P::COLS) {
#pragma unroll
                    for (int a = 0; a < P::NIN; ++a) v[a] = sm->u.f.in[a][b][j * CP + lane];
                    if constexpr (P::NEIGH) {
                        const float sh = __shfl_down_sync(0xffffffffu, v[0], 1);
                        xr = (lane == WARP - 1) ? sm->u.f.in[0][b][j * CP + WARP] : sh;
                    }
                } else {
#pragma unroll
                    for (int a = 0; a < P::NIN; ++a) v[a] = pick4(q[a], e);
                }
                float c, w;
                p.unary(v, xr, j, i, n, k, c, w, acc);
                if (i < n) {
                    if constexpr (P::CREC) crec_w[(long long)i * WARP + lane] = c;
                    if (alive) {
                        float lm, hp;
                        if (i == 0) {
                            if (n == 1) {
                                lm = hp = c;
                            } else {
                                dp_first(d, S, 0, c, w, lm, hp);
                            }
                        } else {
                            alive = dp_step(d, S, RING, c, w, (float)(i + 1), lm, hp);
                        }
                        if (alive) {
                            if (i == n - 1) xlast = (n == 1) ? c : 0.5f * (lm + hp);
                            else rec_w[(long long)i * WARP + lane] = make_float2(lm, hp);
                        }
                    }
                }
            }
        }
        __syncwarp();
        b ^= 1;
    }
    cp_async_wait<0>();
    __threadfence_block();
    __syncwarp();

    // ---------------- backward pass ----------------
    const int n_eff = alive ? n : 0;
    float xv = xlast;
    b = 0;
    fill_records(sm, b, nchunks - 1, lane, rec_w, crec_w, n_eff);
    cp_async_commit();
    for (int ch = nchunks - 1; ch >= 0; --ch) {
        if (ch > 0) fill_records(sm, b ^ 1, ch - 1, lane, rec_w, crec_w, n_eff);
        cp_async_commit();
        cp_async_wait<1>();
        __syncwarp();
#pragma unroll 4
        for (int j = CH - 1; j >= 0; --j) {
            const int i = ch * CH + j;
            if (i < n_eff) {
                if (i < n - 1) {
                    const float2 r = sm->u.b.rec[b][j][lane];
                    xv = clip_to(xv, r.x, r.y);
                }
                float cc = 0.f;
                if constexpr (P::CREC) cc = sm->u.b.crec[b][j][lane];
                if constexpr (P::COLS) {
                    p.emit_cols(i, k, xv, cc);
                } else {
                    sm->u.b.out[lane * RP + j] = xv;
                }
            }
        }
        if constexpr (!P::COLS) {
            __syncwarp();
            // rows whose lane overflowed write nothing here: mask them by length
            if (!alive) sm->len[lane] = 0;
            __syncwarp();
#pragma unroll
            for (int o = 0; o < P::NOUT; ++o) flush_outputs(p, sm, ch, lane, warp_chain0, o);
            __syncwarp();
            if (!alive) sm->len[lane] = n;
        }
        __syncwarp();
        b ^= 1;
    }
    cp_async_wait<0>();

    if (!alive) {
        atomicAdd(&hdr->overflowed, 1ull);
        float2 *sp = spill + p.spill_off(k, start);
        solve_chain_global(p, k, start, n, sp, rec_w, crec_w, lane);
    }
    p.finish(acc);
}

}  // namespace tvk
