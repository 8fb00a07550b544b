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

namespace tvk {

constexpr int WARP = 32;
constexpr int CH = 16;  // nodes per staged chunk

// Device error word bits (workspace header).
constexpr int ERR_BAD_CHAIN = 1;

struct WsHeader {
    int status;              // ERR_* bits, sticky until read
    int pad0;
    unsigned long long overflowed;  // chains finished from the global reserve
    unsigned char pad[48];
};
static_assert(sizeof(WsHeader) == 64, "header size");

struct DPState {
    int F, B;           // logical indices of the first and last breakpoint
    float fl, fs;       // cached first entry (lambda, stored slope)
    float bl, bs;       // cached last entry
    float w_prev;       // weight of the edge into the current node
};

template <int RING>
struct RingStore {
    float2 *col;  // &ring[0][lane]
    static constexpr int cap = RING;
    __device__ __forceinline__ float2 ld(int j) const { return col[(j & (RING - 1)) * WARP]; }
    __device__ __forceinline__ void st(int j, float2 e) const { col[(j & (RING - 1)) * WARP] = e; }
};

struct LinearStore {
    float2 *base;  // 2n+2 entries; logical index j at base[j]
    __device__ __forceinline__ float2 ld(int j) const { return base[j]; }
    __device__ __forceinline__ void st(int j, float2 e) const { base[j] = e; }
};

// Node 0: m^_0(z) = z - c_0 has slope 1, so lambda^-_0 = c_0 - w_0, lambda^+_0 = c_0 + w_0.
template <class S>
__device__ __forceinline__ void dp_first(DPState &d, const S &s, int F0, float c0, float w0,
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
// lambda^-; the right scan removes breakpoints with m^_i > w_i (only among those
// the left scan kept) and places lambda^+. Returns false, leaving the store and
// state untouched, if the new sequence would exceed `cap` entries.
template <class S>
__device__ __forceinline__ bool dp_step(DPState &d, const S &s, int cap, float ci, float wi,
                                        float abar, float &lm, float &hp)
{
    // Left scan: value at the first breakpoint, then the forward recursion.
    float v = d.fl - ci - d.w_prev;
    int last_popped;
    float lm_s;
    if (v >= -wi) {
        last_popped = d.F - 1;  // nothing removed; lambda^- on the left end segment (slope 1)
        lm = d.fl - (v + wi);
        lm_s = 1.f - abar;
    } else {
        int p = d.F;
        float pl = d.fl, ps = d.fs;
        while (p < d.B) {
            float2 q = (p + 1 == d.B) ? make_float2(d.bl, d.bs) : s.ld(p + 1);
            float vq = v + (ps + abar) * (q.x - pl);
            if (vq < -wi) {
                ++p;
                pl = q.x;
                ps = q.y;
                v = vq;
            } else {
                break;
            }
        }
        // Both end values of m^_i are known exactly (-w_{i-1} + lambda_F - c_i at the
        // first breakpoint, w_{i-1} + lambda_B - c_i at the last one). When the scan
        // stopped nearer the last breakpoint, re-evaluate m^_i(lambda_p) by the
        // backward recursion from there: the same value in exact arithmetic, but
        // FP32 rounding of the breakpoints is no longer multiplied by the large
        // slopes of the segments crossed. The walk is shorter than the one just
        // made, so the update stays O(d_i + 1).
        if (d.B - p < p - d.F) {
            float vb = d.bl - ci + d.w_prev;
            float ql = d.bl;
            for (int q = d.B - 1; q >= p; --q) {
                const float2 e = (q == d.F) ? make_float2(d.fl, d.fs) : s.ld(q);
                vb -= (e.y + abar) * (ql - e.x);
                ql = e.x;
            }
            v = vb;
        }
        last_popped = p;
        lm = pl + (-wi - v) / (ps + abar);
        lm_s = ps;  // lambda^- splits old segment p, whose slope it keeps
    }
    // Right scan over the kept breakpoints (index > last_popped).
    int new_last;
    if (d.B > last_popped) {
        float vr = d.bl - ci + d.w_prev;
        if (vr <= wi) {
            hp = d.bl + (wi - vr);  // lambda^+ on the right end segment (slope 1)
            new_last = d.B;
        } else {
            int q = d.B;
            float ql = d.bl;
            for (;;) {
                if (q - 1 > last_popped) {
                    float2 e = (q - 1 == d.F) ? make_float2(d.fl, d.fs) : s.ld(q - 1);
                    float slope = e.y + abar;
                    float vp = vr - slope * (ql - e.x);
                    if (vp > wi) {
                        --q;
                        ql = e.x;
                        vr = vp;
                        continue;
                    }
                    if (q - d.F < d.B - q) {
                        // nearer the first breakpoint: forward recursion from there
                        // (the mirror image of the re-evaluation in the left scan)
                        float vf = d.fl - ci - d.w_prev;
                        float pl = d.fl, ps = d.fs;
                        for (int t = d.F + 1; t <= q; ++t) {
                            const float2 e2 = (t == d.B) ? make_float2(d.bl, d.bs) : s.ld(t);
                            vf += (ps + abar) * (e2.x - pl);
                            pl = e2.x;
                            ps = e2.y;
                        }
                        vr = vf;
                    }
                    hp = ql - (vr - wi) / slope;
                } else {
                    // lambda^+ on the segment that starts at the new lambda^-, where
                    // m^_i = -w_i exactly
                    hp = lm + (wi + wi) / (lm_s + abar);
                }
                break;
            }
            new_last = q - 1;
        }
    } else {
        hp = lm + (wi + wi) / (lm_s + abar);  // every old breakpoint removed on the left
        new_last = last_popped;
    }
    const int nF = last_popped;
    const int nB = (new_last > nF ? new_last : nF) + 1;
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
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ------------------------------------------------------------ warp machinery --
//
// A phase policy P describes one batch of chains and what surrounds the DP:
//   static constexpr bool COLS   chains are columns of a row-major array
//                                (node i of chain k at i*ld + k), else contiguous rows
//   static constexpr int  NIN    number of staged per-node input arrays
//   static constexpr bool NEIGH  also stage input 0 of the column to the right (COLS only)
//   static constexpr bool CREC   record c_i for the epilogue
//   static constexpr int  NOUT   number of row-layout outputs (rows only)
//   active(), num_chains(), max_len()
//   chain(k, &start, &n)         node-0 element offset and length; false => malformed
//   in_ptr(a), in_off(a, k, start), in_lim(a, n), in_ld(a)
//   unary(in[], nb, i, n, k, &c, &w, acc)   c_i and w_i (edge i -> i+1) from staged values
//   unary_direct(i, n, k, start, &c, &w)    the same from global memory (overflow path)
//   emit_cols(i, k, xhat, c)                column-layout output of node i
//   out_ptr(o), out_off(o, k, start), out_val(o, xhat, c)   row-layout outputs
//   finish(acc)                  end-of-thread hook (gap partials)

template <class P, int RING>
struct WarpSmem {
    float in[P::NIN][2][WARP + (P::NEIGH ? 1 : 0)][CH + 1];
    float2 rec[2][CH][WARP];
    float crec[P::CREC ? 2 : 1][P::CREC ? CH : 1][WARP];
    float out[P::COLS ? 1 : WARP][P::COLS ? 1 : CH + 1];
    float2 ring[RING][WARP];
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
        if constexpr (P::COLS) {
            const long long k = warp_chain0 + lane;
            const long long ld = p.in_ld(a);
            const int lim = p.in_lim(a, p.max_len());
            if (k < p.in_kmax(a)) {
#pragma unroll 4
                for (int u = 0; u < CH; ++u) {
                    const int i = chunk * CH + u;
                    if (i < lim) cp_async4(&sm->in[a][b][lane][u], src + (long long)i * ld + k);
                }
            }
            if (P::NEIGH && a == 0 && lane < CH) {
                const long long kn = warp_chain0 + WARP;
                const int i = chunk * CH + lane;
                if (kn < p.in_kmax(a) && i < lim)
                    cp_async4(&sm->in[a][b][WARP][lane], src + (long long)i * ld + kn);
            }
        } else {
#pragma unroll 4
            for (int u = 0; u < CH; ++u) {
                const int t = u * WARP + lane;
                const int jj = t / CH, node = t % CH;
                const int i = chunk * CH + node;
                const int n = sm->len[jj];
                if (i < p.in_lim(a, n))
                    cp_async4(&sm->in[a][b][jj][node],
                              src + p.in_off(a, warp_chain0 + jj, sm->start[jj]) + i);
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
            cp_async8(&sm->rec[b][u][lane], rec_w + (long long)i * WARP + lane);
            if constexpr (P::CREC)
                cp_async4(&sm->crec[b][u][lane], crec_w + (long long)i * WARP + lane);
        }
    }
}

template <class P, int RING>
__device__ __forceinline__ void flush_outputs(const P &p, WarpSmem<P, RING> *sm, int chunk,
                                              int lane, long long warp_chain0, int o)
{
    float *dst = p.out_ptr(o);
#pragma unroll 4
    for (int u = 0; u < CH; ++u) {
        const int t = u * WARP + lane;
        const int jj = t / CH, node = t % CH;
        const int i = chunk * CH + node;
        if (i < sm->len[jj])
            dst[p.out_off(o, warp_chain0 + jj, sm->start[jj]) + i] = sm->out[jj][node];
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
            float2 r = rec_w[(long long)i * WARP + lane];
            xv = clip_to(xv, r.x, r.y);
        }
        p.emit_direct(i, k, start, xv, cc);
    }
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
    float2 *rec_w = rec + wg * (long long)max_len * WARP;
    float *crec_w = P::CREC ? crec + wg * (long long)max_len * WARP : nullptr;

    RingStore<RING> S{&sm->ring[0][lane]};
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
        for (int j = 0; j < CH; ++j) {
            const int i = ch * CH + j;
            float c, w;
            p.unary(sm->in, b, j, lane, i, n, k, c, w, acc);
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
#pragma unroll 1
        for (int j = CH - 1; j >= 0; --j) {
            const int i = ch * CH + j;
            if (i < n_eff) {
                if (i < n - 1) {
                    const float2 r = sm->rec[b][j][lane];
                    xv = clip_to(xv, r.x, r.y);
                }
                float cc = 0.f;
                if constexpr (P::CREC) cc = sm->crec[b][j][lane];
                if constexpr (P::COLS) {
                    p.emit_cols(i, k, xv, cc);
                } else {
                    sm->out[lane][j] = xv;
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
