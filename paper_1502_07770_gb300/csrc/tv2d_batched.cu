// Batched 2D TV-l2 (ROF) denoising of images of uneven size.
//
// Every image runs its own copy of the accelerated primal-dual iteration eq. pd
// (Sec. 6.1) with its own stopping test; the step-size schedule (tau_0 = sigma_0
// = 1, gamma = 1) does not depend on the image, so all images share it. Each
// phase of an iteration is ONE persistent launch over the chains of all images
// still running: warps take chains (one warp per chain, tv_coop.cuh) from an
// atomic work counter, longest chains first. A gap launch tiles all images; the
// last block of each image finalises its gap, iteration count and stop flag, and
// the last block overall decides whether another iteration is needed. The outer
// loop is a CUDA graph with a conditional WHILE node whose body is one iteration
// (column phase, row phase, gap), so the whole solve is one graph launch; where
// conditional nodes are unavailable the same body is replayed from the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "tv2d_common.cuh"
#include "tv_halves.cuh"
#include "tv_launch.cuh"

using namespace tvk;
using namespace tvh;

namespace {

struct BImg {
    const float *f, *wh, *wv;
    float lam;
    int H, W;
    float *x0, *x1, *y;  // x0: the caller's output; x1, y: workspace
    float2 *rec;
    float *crec;
    float2 *spill;
    double inv_N;
};

struct BState {
    int k;            // completed iterations of this image
    int done;         // 1 converged, 2 stopped at max_iters
    double gap;       // last per-pixel gap
    unsigned ticket;  // gap blocks of this image finished in the running launch
    int ntiles, tile0;  // its gap tiles: tile0 .. tile0 + ntiles - 1
};

struct ChainRef {
    int img, idx;  // image, and its row (row phases) or column (column phase)
};

struct GapTile {
    int img;
    long long first, count;  // pixel range of the image
};

struct BCtl {
    unsigned counter;     // work counter of the running phase
    unsigned gap_ticket;  // gap blocks finished in the running launch
    int active;           // images still iterating
    int iter;             // iterations run
    int max_iters;
    double tol;
};

__global__ void batched_init(BState *st, int n_imgs, BCtl *ctl, int max_iters, double tol,
                             Tv2dParams *prm, ParamChunk chunk, const int *ntiles,
                             const int *tile0)
{
    for (int q = threadIdx.x; q < chunk.count; q += blockDim.x) prm[chunk.first + q] = chunk.p[q];
    if (chunk.first != 0) return;
    for (int m = threadIdx.x; m < n_imgs; m += blockDim.x) {
        st[m].k = 0;
        st[m].done = 0;
        st[m].gap = nan("");
        st[m].ticket = 0;
        st[m].ntiles = ntiles[m];
        st[m].tile0 = tile0[m];
    }
    if (threadIdx.x == 0) {
        ctl->counter = 0;
        ctl->gap_ticket = 0;
        ctl->active = n_imgs;
        ctl->iter = 0;
        ctl->max_iters = max_iters;
        ctl->tol = tol;
    }
}

// ------------------------------------------------------------------ policies --
// PHASE 0: x^0 rows, 1: primal rows, 2: dual columns (same arithmetic as the
// single-image policies, with weights present or absent per image at run time).
template <int PHASE>
struct BPol {
    static constexpr bool CREC = PHASE == 2;
    struct Raw {
        float a, b, c, w;
    };
    struct Acc {};
    const BImg *im;
    const float *xin;
    float *xout;
    float ca, cb, sigma, inv_sigma, theta;

    __device__ void setup(const BImg *img, const BState &st, const Tv2dParams *prm)
    {
        im = img;
        const int k = st.k;
        if (PHASE == 1) {
            xin = (k & 1) ? im->x1 : im->x0;
            xout = (k & 1) ? im->x0 : im->x1;
            const double tau = prm[k].tau;
            ca = (float)(tau / (tau + 1.0));
            cb = (float)(1.0 / (tau + 1.0));
        } else if (PHASE == 2) {
            xin = (k & 1) ? im->x1 : im->x0;   // x^k
            xout = (k & 1) ? im->x0 : im->x1;  // x^{k-1}
            sigma = (float)prm[k].sigma;
            inv_sigma = (float)(1.0 / prm[k].sigma);
            theta = (float)prm[k].theta_prev;
        }
    }
    __device__ int max_len() const { return PHASE == 2 ? im->H : im->W; }
    __device__ long long spill_off(long long k, long long) const
    {
        return PHASE == 2 ? k * (2LL * im->H + 2) : k * (2LL * im->W + 2);
    }
    __device__ void fetch(long long k, long long start, int n, int i, Raw &r) const
    {
        const bool in = i < n;
        if (PHASE == 2) {
            const long long o = (long long)i * im->W + k;
            r.a = in ? xin[o] : 0.f;
            r.b = in ? xout[o] : 0.f;
            r.c = in ? im->y[o] : 0.f;
            r.w = (im->wv && i < n - 1) ? im->wv[o] : im->lam;
        } else {
            r.a = in ? im->f[start + i] : 0.f;
            r.b = in ? im->y[start + i] : 0.f;
            r.c = (PHASE == 1 && in) ? xin[start + i] : 0.f;
            r.w = (im->wh && i < n - 1) ? im->wh[k * (im->W - 1) + i] : im->lam;
        }
    }
    __device__ void unary(long long, long long, int, int, const Raw &r, float &c, float &w,
                          Acc &) const
    {
        if (PHASE == 0) {
            c = r.a - r.b;
            w = r.w;
        } else if (PHASE == 1) {
            c = ca * (r.a - r.b) + cb * r.c;
            w = ca * r.w;
        } else {
            c = r.c * inv_sigma + (r.a + theta * (r.a - r.b));
            w = r.w * inv_sigma;
        }
    }
    __device__ void emit(long long k, long long start, int i, float xv, float c) const
    {
        if (PHASE == 0) {
            im->x0[start + i] = xv;
            im->x1[start + i] = xv;
        } else if (PHASE == 1) {
            xout[start + i] = xv;
        } else {
            im->y[(long long)i * im->W + k] = sigma * (c - xv);
        }
    }
    __device__ void unary_direct(int i, int n, long long k, long long start, float &c,
                                 float &w) const
    {
        Raw r;
        fetch(k, start, n, i, r);
        Acc a;
        unary(k, start, n, i, r, c, w, a);
        if (i == n - 1) w = 0.f;
    }
    __device__ void emit_direct(int i, long long k, long long start, float xv, float c) const
    {
        emit(k, start, i, xv, c);
    }
};

constexpr int kBatchedSmemNodes = 2048;

template <int PHASE>
__global__ void __launch_bounds__(256)
    batched_phase_kernel(const BImg *imgs, const BState *st, const ChainRef *chains, int nchains,
                         const Tv2dParams *prm, BCtl *ctl, WsHeader *hdr, int smem_nodes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & (WARP - 1);
    const int warp = threadIdx.x / WARP;
    const int wpb = blockDim.x / WARP;
    float2 *sm_rec = reinterpret_cast<float2 *>(smem_raw) + (size_t)warp * smem_nodes;
    float *sm_crec = reinterpret_cast<float *>(reinterpret_cast<float2 *>(smem_raw) +
                                               (size_t)wpb * smem_nodes) +
                     (size_t)warp * smem_nodes;
    for (;;) {
        int q = 0;
        if (lane == 0) q = (int)atomicAdd(&ctl->counter, 1u);
        q = __shfl_sync(FULL, q, 0);
        if (q >= nchains) break;
        const ChainRef ref = chains[q];
        const BImg *im = imgs + ref.img;
        if (PHASE != 0 && st[ref.img].done) continue;
        BPol<PHASE> p;
        p.setup(im, st[ref.img], prm);
        const int n = PHASE == 2 ? im->H : im->W;
        const long long start = PHASE == 2 ? ref.idx : (long long)ref.idx * im->W;
        typename BPol<PHASE>::Acc acc;
        coop_solve_chain(p, acc, ref.idx, start, n, lane, sm_rec, sm_crec, smem_nodes, im->rec,
                         im->crec, im->spill + p.spill_off(ref.idx, start), hdr);
    }
}

// ------------------------------------------------ one thread per chain ------
// Large batches: a warp takes a group of up to 32 consecutive rows (or columns) of
// one image and runs the one-thread-per-chain dynamic program of tv_dp.cuh on them;
// the groups of all images form one launch per phase (longest chains first).
// Records of a group: 32 slots x its chain length, from the group's rec0.
struct BGroup {
    int img, first, count, pad;
    long long rec0;
};

constexpr int kBRing = 32;

__device__ __forceinline__ bool al16(const void *q) { return ((uintptr_t)q & 15) == 0; }

template <int PHASE>  // 0: x^0 rows, 1: primal rows
struct BRowsTP {
    static constexpr bool COLS = false;
    static constexpr int NIN = PHASE == 0 ? 3 : 4;  // f, y, (x^k), w_h
    static constexpr int WI = NIN - 1;              // the weights input
    static constexpr bool NEIGH = false;
    static constexpr bool CREC = false;
    static constexpr int NOUT = PHASE == 0 ? 2 : 1;
    struct Acc {};
    const BImg *imgs;
    const BState *st;
    const BGroup *groups;
    long long nslots;
    int maxlen;
    int cpw_log;  // log2 of the chains per warp (5: one thread per chain, 4: per half)
    const Tv2dParams *prm;
    const float2 *spill_base;
    // bound per warp
    const BImg *im;
    int r0, cnt;
    long long rec0;
    const float *xin;
    float *xout;
    float ca, cb;
    bool vec, vecw;

    __device__ bool resolve() { return true; }
    __device__ long long num_chains() const { return nslots; }
    __device__ int max_len() const { return maxlen; }
    __device__ bool bind_warp(long long wc0)
    {
        const BGroup g = groups[wc0 >> cpw_log];
        const BState &s = st[g.img];
        if (PHASE != 0 && s.done) return false;
        im = imgs + g.img;
        r0 = g.first;
        cnt = g.count;
        rec0 = g.rec0;
        xin = xout = nullptr;
        ca = cb = 0.f;
        if (PHASE == 1) {
            const int k = s.k;
            xin = (k & 1) ? im->x1 : im->x0;
            xout = (k & 1) ? im->x0 : im->x1;
            const double tau = prm[k].tau;
            ca = (float)(tau / (tau + 1.0));
            cb = (float)(1.0 / (tau + 1.0));
        }
        vec = im->W % 4 == 0 && al16(im->f) && al16(im->y) && al16(im->x0) && al16(im->x1);
        vecw = im->wh != nullptr && (im->W - 1) % 4 == 0 && al16(im->wh);
        return true;
    }
    __device__ long long rec_slot(long long, int) const { return rec0; }
    __device__ int row_of(long long k) const { return r0 + (int)(k & ((1 << cpw_log) - 1)); }
    __device__ bool chain(long long k, long long &start, int &n) const
    {
        start = 0;
        n = 0;
        if ((int)(k & ((1 << cpw_log) - 1)) < cnt) {
            start = (long long)row_of(k) * im->W;
            n = im->W;
        }
        return true;
    }
    __device__ const float *in_ptr(int a) const
    {
        if (a == 0) return im->f;
        if (a == 1) return im->y;
        if (PHASE == 1 && a == 2) return xin;
        return im->wh;  // may be NULL: lambda then
    }
    __device__ long long in_off(int a, long long k, long long start) const
    {
        return a == WI ? (long long)row_of(k) * (im->W - 1) : start;
    }
    __device__ int in_lim(int a, int n) const { return a == WI ? n - 1 : n; }
    __device__ bool in_vec(int a) const { return a == WI ? vecw : vec; }
    __device__ bool out_vec() const { return vec; }
    __device__ __forceinline__ void unary_vals(float fv, float yv, float xv, float wv, int i, int n,
                                               float &c, float &w) const
    {
        if (PHASE == 0) {
            c = fv - yv;
            w = (i < n - 1) ? wv : 0.f;
        } else {
            c = ca * (fv - yv) + cb * xv;
            w = (i < n - 1) ? ca * wv : 0.f;
        }
    }
    __device__ void unary(const float (&v)[NIN], float, int, int i, int n, long long, float &c,
                          float &w, Acc &) const
    {
        const float wv = im->wh ? v[WI] : im->lam;
        unary_vals(v[0], v[1], PHASE == 1 ? v[2] : 0.f, wv, i, n, c, w);
    }
    __device__ void unary_direct(int i, int n, long long k, long long start, float &c,
                                 float &w) const
    {
        const float wv = (im->wh && i < n - 1) ? im->wh[(long long)row_of(k) * (im->W - 1) + i]
                                               : im->lam;
        unary_vals(im->f[start + i], im->y[start + i], PHASE == 1 ? xin[start + i] : 0.f, wv, i, n,
                   c, w);
    }
    __device__ float *out_ptr(int o) const
    {
        if (PHASE == 0) return o == 0 ? im->x0 : im->x1;
        return xout;
    }
    __device__ long long out_off(int, long long, long long start) const { return start; }
    __device__ void emit_cols(int, long long, float, float) const {}
    __device__ void emit_direct(int i, long long, long long start, float xv, float) const
    {
        if (PHASE == 0) {
            im->x0[start + i] = xv;
            im->x1[start + i] = xv;
        } else {
            xout[start + i] = xv;
        }
    }
    __device__ long long spill_off(long long k, long long) const
    {
        return (im->spill - spill_base) + (long long)row_of(k) * (2LL * im->W + 2);
    }
    __device__ void acc_init(Acc &) const {}
    __device__ void finish(Acc &) const {}
    __device__ void finish_empty() const {}
};

// Dual (column) phase.
struct BColsTP {
    static constexpr bool COLS = true;
    static constexpr int NIN = 4;  // x^k, x^{k-1}, y, w_v
    static constexpr int WI = 3;   // the weights input
    static constexpr bool NEIGH = false;
    static constexpr bool CREC = true;
    static constexpr int NOUT = 0;
    struct Acc {};
    const BImg *imgs;
    const BState *st;
    const BGroup *groups;
    long long nslots;
    int maxlen;
    int cpw_log;  // log2 of the chains per warp (5: one thread per chain, 4: per half)
    const Tv2dParams *prm;
    const float2 *spill_base;
    // bound per warp
    const BImg *im;
    int c0, cnt;
    long long rec0;
    const float *xk, *xkm1;
    float sigma, inv_sigma, theta;
    bool vec;

    __device__ bool resolve() { return true; }
    __device__ long long num_chains() const { return nslots; }
    __device__ int max_len() const { return maxlen; }
    __device__ bool bind_warp(long long wc0)
    {
        const BGroup g = groups[wc0 >> cpw_log];
        const BState &s = st[g.img];
        if (s.done) return false;
        im = imgs + g.img;
        c0 = g.first;
        cnt = g.count;
        rec0 = g.rec0;
        const int k = s.k;
        xk = (k & 1) ? im->x1 : im->x0;
        xkm1 = (k & 1) ? im->x0 : im->x1;
        sigma = (float)prm[k].sigma;
        inv_sigma = (float)(1.0 / prm[k].sigma);
        theta = (float)prm[k].theta_prev;
        vec = im->W % 4 == 0 && al16(im->x0) && al16(im->x1) && al16(im->y) &&
              (im->wv == nullptr || al16(im->wv));
        return true;
    }
    __device__ long long col_base(long long) const { return c0; }
    __device__ long long rec_slot(long long, int) const { return rec0; }
    __device__ bool chain(long long k, long long &start, int &n) const
    {
        start = 0;
        n = 0;
        const int l = (int)(k & ((1 << cpw_log) - 1));
        if (l < cnt) {
            start = c0 + l;  // the column
            n = im->H;
        }
        return true;
    }
    __device__ const float *in_ptr(int a) const
    {
        return a == 0 ? xk : (a == 1 ? xkm1 : (a == 2 ? im->y : im->wv));
    }
    __device__ long long in_off(int, long long, long long start) const { return start; }
    __device__ int in_lim(int a, int) const { return a == 3 ? im->H - 1 : im->H; }
    __device__ long long in_ld(int) const { return im->W; }
    __device__ long long in_kmax(int) const { return c0 + cnt; }
    __device__ bool in_vec(int) const { return vec; }
    __device__ bool out_vec() const { return false; }
    __device__ void unary(const float (&v)[NIN], float, int, int i, int n, long long, float &c,
                          float &w, Acc &) const
    {
        const float wvv = im->wv ? v[3] : im->lam;
        c = v[2] * inv_sigma + (v[0] + theta * (v[0] - v[1]));  // eta / sigma
        w = (i < n - 1) ? wvv * inv_sigma : 0.f;
    }
    __device__ void unary_direct(int i, int n, long long, long long col, float &c, float &w) const
    {
        (void)c;  // c comes from the forward-pass record
        const float wvv = (im->wv && i < n - 1) ? im->wv[(long long)i * im->W + col] : im->lam;
        w = (i < n - 1) ? wvv * inv_sigma : 0.f;
    }
    __device__ float *out_ptr(int) const { return nullptr; }
    __device__ long long out_off(int, long long, long long) const { return 0; }
    __device__ void emit_cols(int i, long long k, float xhat, float c) const
    {
        const int l = (int)(k & ((1 << cpw_log) - 1));
        if (l < cnt) im->y[(long long)i * im->W + c0 + l] = sigma * (c - xhat);
    }
    // c_i of column `col` from global memory (the overflow path of the halves kernel)
    __device__ float c_direct(int i, long long, long long col) const
    {
        const long long o = (long long)i * im->W + col;
        return im->y[o] * inv_sigma + (xk[o] + theta * (xk[o] - xkm1[o]));
    }
    __device__ void emit_direct(int i, long long, long long col, float xhat, float c) const
    {
        im->y[(long long)i * im->W + col] = sigma * (c - xhat);
    }
    __device__ long long spill_off(long long, long long col) const
    {
        return (im->spill - spill_base) + col * (2LL * im->H + 2);
    }
    __device__ void acc_init(Acc &) const {}
    __device__ void finish(Acc &) const {}
    __device__ void finish_empty() const {}
};

constexpr int kBGapThreads = 256;
constexpr int kGapBatch = 4;  // pixels of a thread whose loads are in flight together

// No launch bound: one capped the walk at 64 registers (kBGapThreads threads a block).
__global__ void
    batched_gap_kernel(const BImg *imgs, BState *st, const GapTile *tiles, const Tv2dParams *prm,
                       double *partials, BCtl *ctl, cudaGraphConditionalHandle cond, int use_cond)
{
    __shared__ double red[kBGapThreads / WARP];
    __shared__ int last_img;
    const GapTile t = tiles[blockIdx.x];
    const BImg *im = imgs + t.img;
    BState &s = st[t.img];
    const bool run = !s.done;
    double acc = 0.0;
    if (run) {
        const int k = s.k;
        const float *x1 = ((k + 1) & 1) ? im->x1 : im->x0;  // x^{k+1}
        const float *x0 = (k & 1) ? im->x1 : im->x0;        // x^k
        const float inv_tau = (float)(1.0 / prm[k].tau);
        const long long W = im->W, H = im->H;
        float part = 0.f;
        int cnt = 0;
        const float *__restrict__ f = im->f;
        const float *__restrict__ wh = im->wh;
        const float *__restrict__ wv = im->wv;
        const float lam = im->lam;
        // row and column advance incrementally along the block-stride walk; the loads of
        // kGapBatch pixels are issued before any of them is used (memory-level
        // parallelism), and the pixels are summed in walk order as before
        const long long stride = blockDim.x;
        const long long dr = stride / W, dc = stride - dr * W;
        const long long end = t.first + t.count;
        long long q = t.first + threadIdx.x;
        long long r = q / W, c = q - r * W;
        for (; q < end; q += kGapBatch * stride) {
            float xv[kGapBatch], fv[kGapBatch], xp[kGapBatch], xr[kGapBatch], xd[kGapBatch],
                whv[kGapBatch], wvv[kGapBatch];
            bool in[kGapBatch], hr[kGapBatch], hd[kGapBatch];
            long long qj = q;
#pragma unroll
            for (int j = 0; j < kGapBatch; ++j) {
                in[j] = qj < end;
                hr[j] = in[j] && c + 1 < W;
                hd[j] = in[j] && r + 1 < H;
                xv[j] = in[j] ? x1[qj] : 0.f;
                fv[j] = in[j] ? f[qj] : 0.f;
                xp[j] = in[j] ? x0[qj] : 0.f;
                xr[j] = hr[j] ? x1[qj + 1] : 0.f;
                xd[j] = hd[j] ? x1[qj + W] : 0.f;
                whv[j] = hr[j] ? (wh ? wh[r * (W - 1) + c] : lam) : 0.f;
                wvv[j] = hd[j] ? (wv ? wv[qj] : lam) : 0.f;
                qj += stride;
                c += dc;
                r += dr;
                if (c >= W) {
                    c -= W;
                    ++r;
                }
            }
#pragma unroll
            for (int j = 0; j < kGapBatch; ++j) {
                if (!in[j]) continue;
                const float z = xv[j] + (xv[j] - xp[j]) * inv_tau;
                float v = 0.5f * (xv[j] - fv[j]) * (xv[j] - fv[j]) + 0.5f * (z - fv[j]) * (z + fv[j]);
                if (hr[j]) v += whv[j] * fabsf(xr[j] - xv[j]);
                if (hd[j]) v += wvv[j] * fabsf(xd[j] - xv[j]);
                part += v;
                if (++cnt == 32) {
                    acc += (double)part;
                    part = 0.f;
                    cnt = 0;
                }
            }
        }
        acc += (double)part;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & (WARP - 1)) == 0) red[threadIdx.x / WARP] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        last_img = 0;
        if (run) {
            double b = 0.0;
            for (int w = 0; w < kBGapThreads / WARP; ++w) b += red[w];
            partials[blockIdx.x] = b;
            __threadfence();
            if (atomicAdd(&s.ticket, 1u) == (unsigned)s.ntiles - 1) {
                // last block of this image: reduce its tiles in order
                __threadfence();
                double G = 0.0;
                for (int q = s.tile0; q < s.tile0 + s.ntiles; ++q) G += __ldcg(partials + q);
                s.ticket = 0;
                const double g = G * im->inv_N;
                s.gap = g;
                s.k = s.k + 1;
                if (ctl->tol > 0.0 && g <= ctl->tol) {
                    s.done = 1;
                    atomicSub(&ctl->active, 1);
                } else if (s.k >= ctl->max_iters) {
                    s.done = 2;
                    atomicSub(&ctl->active, 1);
                }
            }
        }
        __threadfence();
        if (atomicAdd(&ctl->gap_ticket, 1u) == gridDim.x - 1) {
            __threadfence();
            ctl->gap_ticket = 0;
            ctl->iter = ctl->iter + 1;
            const int more = (ctl->active > 0 && ctl->iter < ctl->max_iters) ? 1 : 0;
            if (use_cond) cudaGraphSetConditional(cond, (unsigned)more);
        }
    }
}

// ---------------------------------------------------------------- host side --
struct Plan {
    std::vector<BImg> imgs;
    std::vector<ChainRef> cols, rows;
    std::vector<BGroup> rgroups, cgroups;  // one-thread-per-chain groups
    bool thread_rows = false, thread_cols = false;
    bool halves = false;  // thread-per-chain batches run a thread per chain half
    std::vector<GapTile> tiles;
    std::vector<int> ntiles, tile0;
    int max_h = 0, max_w = 0;
    int blocks[3] = {1, 1, 1};  // persistent grid of each phase kernel
    int smem_nodes[3] = {0, 0, 0};
};

struct BatchedWs {
    BImg *imgs;
    BState *st;
    ChainRef *cols, *rows;
    BGroup *rgroups, *cgroups;
    float2 *trec;  // records of the one-thread-per-chain launches
    float *tcrec;
    GapTile *tiles;
    int *ntiles, *tile0;
    double *partials;
    Tv2dParams *prm;
    BCtl *ctl;
    WsHeader *hdr;
    size_t bytes;
};

constexpr long long kGapTilePixels = 1 << 14;  // 64 pixels per thread: enough blocks in flight

// Lays out the workspace (base may be NULL to size it) and fills the image table.
BatchedWs carve_batched(void *base, const tv_image_desc *d, int n, int max_iters, Plan &plan)
{
    Carver cv(base);
    BatchedWs o;
    long long ncols = 0, nrows = 0, ntiles = 0, nrg = 0, ncg = 0, rrec = 0, crec = 0;
    for (int m = 0; m < n; ++m) {
        ncols += d[m].W;
        nrows += d[m].H;
        ntiles += (d[m].H * d[m].W + kGapTilePixels - 1) / kGapTilePixels;
        // groups of 32 chains (a thread per chain) or of 16 (a thread per chain half):
        // room for either layout of the records
        const long long rg = (d[m].H + WARP - 1) / WARP, cg = (d[m].W + WARP - 1) / WARP;
        const long long rg2 = (d[m].H + HW - 1) / HW, cg2 = (d[m].W + HW - 1) / HW;
        nrg += rg2;
        ncg += cg2;
        rrec += std::max(rg * WARP * d[m].W, rg2 * WARP * ((d[m].W + 1) / 2));
        crec += std::max(cg * WARP * d[m].H, cg2 * WARP * ((d[m].H + 1) / 2));
    }
    o.imgs = cv.take<BImg>((size_t)n);
    o.st = cv.take<BState>((size_t)n);
    o.cols = cv.take<ChainRef>((size_t)ncols);
    o.rows = cv.take<ChainRef>((size_t)nrows);
    o.tiles = cv.take<GapTile>((size_t)ntiles);
    o.rgroups = cv.take<BGroup>((size_t)nrg);
    o.cgroups = cv.take<BGroup>((size_t)ncg);
    o.trec = cv.take<float2>((size_t)std::max(rrec, crec));
    o.tcrec = cv.take<float>((size_t)crec);
    o.ntiles = cv.take<int>((size_t)n);
    o.tile0 = cv.take<int>((size_t)n);
    o.partials = cv.take<double>((size_t)ntiles);
    o.prm = cv.take<Tv2dParams>((size_t)max_iters + 2);
    o.ctl = cv.take<BCtl>(1);
    o.hdr = cv.take<WsHeader>(1);
    plan.imgs.resize(n);
    for (int m = 0; m < n; ++m) {
        const long long H = d[m].H, W = d[m].W, N = H * W;
        BImg &b = plan.imgs[m];
        b.f = d[m].img;
        b.wh = d[m].wh;
        b.wv = d[m].wv;
        b.lam = d[m].lambda;
        b.H = (int)H;
        b.W = (int)W;
        b.x0 = d[m].x;
        b.x1 = cv.take<float>((size_t)N);
        b.y = cv.take<float>((size_t)N);
        b.rec = cv.take<float2>((size_t)N);
        b.crec = cv.take<float>((size_t)N);
        const long long sp = std::max(H * (2 * W + 2), W * (2 * H + 2));
        b.spill = cv.take<float2>((size_t)sp);
        b.inv_N = 1.0 / (double)N;
    }
    o.bytes = align_up(cv.used, 256);
    return o;
}

void build_plan(const tv_image_desc *d, int n, Plan &plan)
{
    std::vector<int> by_h(n), by_w(n);
    for (int m = 0; m < n; ++m) by_h[m] = by_w[m] = m;
    // longest chains first: columns have H nodes, rows W nodes
    std::stable_sort(by_h.begin(), by_h.end(), [&](int a, int b) { return d[a].H > d[b].H; });
    std::stable_sort(by_w.begin(), by_w.end(), [&](int a, int b) { return d[a].W > d[b].W; });
    plan.cols.clear();
    plan.rows.clear();
    for (int m : by_h)
        for (int c = 0; c < d[m].W; ++c) plan.cols.push_back(ChainRef{m, c});
    for (int m : by_w)
        for (int r = 0; r < d[m].H; ++r) plan.rows.push_back(ChainRef{m, r});
    plan.rgroups.clear();
    plan.cgroups.clear();
    // a thread per chain half (16 chains per warp, ceil(len / 2) record rows) or a
    // thread per chain (32 chains per warp, len record rows)
    plan.halves = thread_split() != 0;
    const int G = plan.halves ? HW : WARP;
    long long rrec = 0, crec = 0;
    for (int m : by_w)
        for (long long r = 0; r < d[m].H; r += G) {
            plan.rgroups.push_back(
                BGroup{m, (int)r, (int)std::min<long long>(G, d[m].H - r), 0, rrec});
            rrec += (long long)WARP * (plan.halves ? (d[m].W + 1) / 2 : d[m].W);
        }
    for (int m : by_h)
        for (long long c = 0; c < d[m].W; c += G) {
            plan.cgroups.push_back(
                BGroup{m, (int)c, (int)std::min<long long>(G, d[m].W - c), 0, crec});
            crec += (long long)WARP * (plan.halves ? (d[m].H + 1) / 2 : d[m].H);
        }
    // batches larger than the warp-per-chain limit run one thread per chain
    plan.thread_rows = (long long)plan.rows.size() > coop_max_chains();
    plan.thread_cols = (long long)plan.cols.size() > coop_max_chains();
    plan.tiles.clear();
    plan.ntiles.assign(n, 0);
    plan.tile0.assign(n, 0);
    plan.max_h = plan.max_w = 0;
    for (int m = 0; m < n; ++m) {
        const long long N = d[m].H * d[m].W;
        plan.tile0[m] = (int)plan.tiles.size();
        for (long long first = 0; first < N; first += kGapTilePixels) {
            plan.tiles.push_back(GapTile{m, first, std::min(kGapTilePixels, N - first)});
            plan.ntiles[m] += 1;
        }
        plan.max_h = std::max(plan.max_h, (int)d[m].H);
        plan.max_w = std::max(plan.max_w, (int)d[m].W);
    }
}

int g_batched_wpb = 4;  // warps per block of the phase kernels (tunable)

template <int PHASE>
size_t phase_smem(int smem_nodes)
{
    return (size_t)g_batched_wpb * smem_nodes * (sizeof(float2) + (PHASE == 2 ? sizeof(float) : 0));
}

// Host set-up of one phase kernel (shared memory opt-in, persistent grid size),
// done before any capture.
template <int PHASE>
tv_status prepare_phase(Plan &plan, int nchains, int max_len)
{
    const int wpb = g_batched_wpb;
    const int nodes = (max_len <= kBatchedSmemNodes &&
                       phase_smem<PHASE>(kBatchedSmemNodes) <= (size_t)200 * 1024)
                          ? kBatchedSmemNodes
                          : 0;
    const size_t smem = phase_smem<PHASE>(nodes);
    tv_status st = check_cuda(cudaFuncSetAttribute(batched_phase_kernel<PHASE>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem),
                              "cudaFuncSetAttribute");
    if (st != TV_OK) return st;
    int per_sm = 0;
    st = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                        &per_sm, batched_phase_kernel<PHASE>, wpb * WARP, smem),
                    "occupancy");
    if (st != TV_OK) return st;
    long long blocks = (long long)(per_sm < 1 ? 1 : per_sm) * sm_count_current();
    const long long need = (nchains + wpb - 1) / wpb;
    if (blocks > need) blocks = need;
    plan.blocks[PHASE] = (int)(blocks < 1 ? 1 : blocks);
    plan.smem_nodes[PHASE] = nodes;
    return TV_OK;
}

template <int PHASE>
tv_status launch_phase(const BatchedWs &ws, const Plan &plan, const ChainRef *chains, int nchains,
                       cudaStream_t s)
{
    tv_status st = check_cuda(cudaMemsetAsync(&ws.ctl->counter, 0, sizeof(unsigned), s),
                              "reset work counter");
    if (st != TV_OK) return st;
    batched_phase_kernel<PHASE><<<(unsigned)plan.blocks[PHASE], g_batched_wpb * WARP,
                                  phase_smem<PHASE>(plan.smem_nodes[PHASE]), s>>>(
        ws.imgs, ws.st, chains, nchains, ws.prm, ws.ctl, ws.hdr, plan.smem_nodes[PHASE]);
    return check_cuda(cudaGetLastError(), "batched phase launch");
}

constexpr int kBRingHalf = 16;  // ring entries per chain half

template <class P>
P thread_policy(const BatchedWs &ws, const Plan &plan, bool cols)
{
    P p{};
    p.imgs = ws.imgs;
    p.st = ws.st;
    p.groups = cols ? ws.cgroups : ws.rgroups;
    p.cpw_log = plan.halves ? 4 : 5;
    p.nslots = (long long)(cols ? plan.cgroups.size() : plan.rgroups.size()) << p.cpw_log;
    p.maxlen = cols ? plan.max_h : plan.max_w;
    p.prm = ws.prm;
    p.spill_base = plan.imgs[0].spill;
    return p;
}

template <class P>
tv_status prepare_thread()
{
    tv_status st = check_cuda(cudaFuncSetAttribute(chain_batch_kernel<P, kBRing>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)(4 * sizeof(WarpSmem<P, kBRing>))),
                              "cudaFuncSetAttribute");
    if (st != TV_OK) return st;
    return check_cuda(cudaFuncSetAttribute(chain_halves_kernel<P, kBRingHalf>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(4 * sizeof(HalfSmem<P, kBRingHalf>))),
                      "cudaFuncSetAttribute");
}

template <class P>
tv_status launch_thread(const BatchedWs &ws, const Plan &plan, bool cols, cudaStream_t s)
{
    const P p = thread_policy<P>(ws, plan, cols);
    if (plan.halves) {
        const Shape sh = chains_shape(p.nslots / HW, (const void *)chain_halves_kernel<P, kBRingHalf>,
                                      sizeof(HalfSmem<P, kBRingHalf>));
        chain_halves_kernel<P, kBRingHalf><<<(unsigned)sh.blocks, sh.wpb * WARP,
                                             sh.wpb * sizeof(HalfSmem<P, kBRingHalf>), s>>>(
            p, ws.trec, ws.tcrec, const_cast<float2 *>(p.spill_base), ws.hdr, 0);
        return check_cuda(cudaGetLastError(), "batched thread-per-half launch");
    }
    const Shape sh = chains_shape(p.nslots / WARP, (const void *)chain_batch_kernel<P, kBRing>,
                                  sizeof(WarpSmem<P, kBRing>));
    chain_batch_kernel<P, kBRing><<<(unsigned)sh.blocks, sh.wpb * WARP,
                                    sh.wpb * sizeof(WarpSmem<P, kBRing>), s>>>(
        p, ws.trec, ws.tcrec, const_cast<float2 *>(p.spill_base), ws.hdr);
    return check_cuda(cudaGetLastError(), "batched thread-per-chain launch");
}

tv_status launch_iteration(const BatchedWs &ws, const Plan &plan, cudaStream_t s,
                           cudaGraphConditionalHandle cond, int use_cond)
{
    tv_status st = plan.thread_cols ? launch_thread<BColsTP>(ws, plan, true, s)
                                    : launch_phase<2>(ws, plan, ws.cols, (int)plan.cols.size(), s);
    if (st != TV_OK) return st;
    st = plan.thread_rows ? launch_thread<BRowsTP<1>>(ws, plan, false, s)
                          : launch_phase<1>(ws, plan, ws.rows, (int)plan.rows.size(), s);
    if (st != TV_OK) return st;
    batched_gap_kernel<<<(unsigned)plan.tiles.size(), kBGapThreads, 0, s>>>(
        ws.imgs, ws.st, ws.tiles, ws.prm, ws.partials, ws.ctl, cond, use_cond);
    return check_cuda(cudaGetLastError(), "batched gap launch");
}

template <class T>
tv_status upload(T *dst, const std::vector<T> &src, cudaStream_t s)
{
    if (src.empty()) return TV_OK;
    return check_cuda(cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(),
                                      cudaMemcpyHostToDevice, s),
                      "upload batch tables");
}

std::mutex g_capture_mu;
cudaStream_t g_capture_stream = nullptr;
thread_local int g_last_graphed = -1;
// 1: run the outer loop as a conditional graph when available; 0: always replay it
// from the host. Initial value from TV_BATCHED_GRAPH ("0" disables the graph).
std::atomic<int> g_graph_mode{-1};

bool graph_mode_on()
{
    int m = g_graph_mode.load();
    if (m < 0) {
        const char *e = std::getenv("TV_BATCHED_GRAPH");
        m = (e && e[0] == '0') ? 0 : 1;
        g_graph_mode.store(m);
    }
    return m == 1;
}

}  // namespace

extern "C" {

size_t tv2d_batched_workspace_size(const tv_image_desc *imgs, int n_imgs, int max_iters)
{
    if (!imgs || n_imgs < 1 || max_iters < 0) return 0;
    for (int m = 0; m < n_imgs; ++m)
        if (imgs[m].H < 1 || imgs[m].W < 1) return 0;
    Plan plan;
    return carve_batched(nullptr, imgs, n_imgs, max_iters, plan).bytes;
}

int tv2d_batched_last_mode(void) { return g_last_graphed; }

tv_status tv_set_batched_graph(int on)
{
    clear_error();
    if (on != 0 && on != 1) {
        set_error("tv_set_batched_graph: 0 or 1");
        return TV_ERR_INVALID;
    }
    g_graph_mode.store(on);
    return TV_OK;
}

tv_status tv_set_batched_warps(int warps_per_block)
{
    clear_error();
    if (warps_per_block != 1 && warps_per_block != 2 && warps_per_block != 4 &&
        warps_per_block != 8) {
        set_error("tv_set_batched_warps: 1, 2, 4 or 8");
        return TV_ERR_INVALID;
    }
    g_batched_wpb = warps_per_block;
    return TV_OK;
}

tv_status tv2d_denoise_batched(const tv_image_desc *imgs, int n_imgs, int max_iters,
                               double gap_tol, int *iters_out, double *gap_out, void *d_workspace,
                               size_t workspace_bytes, tv_stream_t stream)
{
    clear_error();
    if (!imgs || n_imgs < 1 || max_iters < 0 || max_iters > (1 << 24) || !d_workspace) {
        set_error("tv2d_denoise_batched: need images, n_imgs >= 1, 0 <= max_iters and a workspace");
        return TV_ERR_INVALID;
    }
    if (!(gap_tol >= 0.0 && gap_tol < INFINITY)) {
        set_error("tv2d_denoise_batched: gap_tol must be finite and >= 0");
        return TV_ERR_INVALID;
    }
    for (int m = 0; m < n_imgs; ++m) {
        const tv_image_desc &d = imgs[m];
        if (!d.img || !d.x || d.H < 1 || d.W < 1 || d.H > (1 << 20) || d.W > (1 << 20) ||
            d.H * d.W > (1LL << 31)) {
            set_error("tv2d_denoise_batched: image %d: need img, x and 1 <= H, W", m);
            return TV_ERR_INVALID;
        }
        if ((!d.wh || !d.wv) && !(d.lambda >= 0.f && d.lambda < INFINITY)) {
            set_error("tv2d_denoise_batched: image %d: lambda must be finite and >= 0", m);
            return TV_ERR_INVALID;
        }
        if (d.x == d.img || (d.y0 && d.x == d.y0)) {
            set_error("tv2d_denoise_batched: image %d: x must not alias the inputs", m);
            return TV_ERR_INVALID;
        }
    }
    Plan plan;
    BatchedWs ws = carve_batched(d_workspace, imgs, n_imgs, max_iters, plan);
    if (workspace_bytes < ws.bytes) {
        set_error("tv2d_denoise_batched: workspace of %zu bytes, %zu needed", workspace_bytes,
                  ws.bytes);
        return TV_ERR_NOMEM;
    }
    build_plan(imgs, n_imgs, plan);
    cudaStream_t s = (cudaStream_t)stream;
    tv_status st;
    if ((st = upload(ws.imgs, plan.imgs, s)) != TV_OK) return st;
    if ((st = upload(ws.cols, plan.cols, s)) != TV_OK) return st;
    if ((st = upload(ws.rows, plan.rows, s)) != TV_OK) return st;
    if ((st = upload(ws.tiles, plan.tiles, s)) != TV_OK) return st;
    if ((st = upload(ws.ntiles, plan.ntiles, s)) != TV_OK) return st;
    if ((st = upload(ws.tile0, plan.tile0, s)) != TV_OK) return st;
    if ((st = prepare_phase<0>(plan, (int)plan.rows.size(), plan.max_w)) != TV_OK) return st;
    if ((st = prepare_phase<1>(plan, (int)plan.rows.size(), plan.max_w)) != TV_OK) return st;
    if ((st = prepare_phase<2>(plan, (int)plan.cols.size(), plan.max_h)) != TV_OK) return st;
    if ((st = upload(ws.rgroups, plan.rgroups, s)) != TV_OK) return st;
    if ((st = upload(ws.cgroups, plan.cgroups, s)) != TV_OK) return st;
    if ((st = prepare_thread<BRowsTP<0>>()) != TV_OK) return st;
    if ((st = prepare_thread<BRowsTP<1>>()) != TV_OK) return st;
    if ((st = prepare_thread<BColsTP>()) != TV_OK) return st;
    {
        static thread_local ParamChunk chunk;
        for (int first = 0; first <= max_iters; first += kParamChunk) {
            fill_params(chunk, first, std::min(kParamChunk, max_iters + 1 - first));
            batched_init<<<1, 128, 0, s>>>(ws.st, n_imgs, ws.ctl, max_iters, gap_tol, ws.prm, chunk,
                                           ws.ntiles, ws.tile0);
            if ((st = check_cuda(cudaGetLastError(), "batched init")) != TV_OK) return st;
            note_launch();
        }
    }
    if ((st = check_cuda(cudaMemsetAsync(ws.hdr, 0, sizeof(WsHeader), s), "memset")) != TV_OK)
        return st;
    for (int m = 0; m < n_imgs; ++m) {
        const size_t bytes = sizeof(float) * (size_t)(imgs[m].H * imgs[m].W);
        st = imgs[m].y0 ? check_cuda(cudaMemcpyAsync(plan.imgs[m].y, imgs[m].y0, bytes,
                                                     cudaMemcpyDeviceToDevice, s), "copy y0")
                        : check_cuda(cudaMemsetAsync(plan.imgs[m].y, 0, bytes, s), "zero y");
        if (st != TV_OK) return st;
    }
    st = plan.thread_rows ? launch_thread<BRowsTP<0>>(ws, plan, false, s)
                          : launch_phase<0>(ws, plan, ws.rows, (int)plan.rows.size(), s);
    if (st != TV_OK) return st;
    note_launch();

    if (max_iters > 0) {
        // The outer loop as one graph: a WHILE node whose body is one iteration.
        bool graphed = false;
        if (!graph_mode_on()) {
            g_last_graphed = 0;
        } else {
            std::lock_guard<std::mutex> lk(g_capture_mu);
            if (!g_capture_stream)
                cudaStreamCreateWithFlags(&g_capture_stream, cudaStreamNonBlocking);
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            cudaGraphConditionalHandle cond;
            cudaGraphNodeParams cp = {};
            cudaGraphNode_t cnode;
            bool ok = g_capture_stream && cudaGraphCreate(&graph, 0) == cudaSuccess &&
                      cudaGraphConditionalHandleCreate(&cond, graph, 1,
                                                       cudaGraphCondAssignDefault) == cudaSuccess;
            if (ok) {
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = cond;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                ok = cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp) == cudaSuccess;
            }
            if (ok) {
                cudaGraph_t body = cp.conditional.phGraph_out[0];
                ok = cudaStreamBeginCaptureToGraph(g_capture_stream, body, nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                if (ok) {
                    const tv_status lst = launch_iteration(ws, plan, g_capture_stream, cond, 1);
                    cudaGraph_t captured = nullptr;
                    ok = cudaStreamEndCapture(g_capture_stream, &captured) == cudaSuccess &&
                         lst == TV_OK;
                }
            }
            if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
            if (ok) ok = cudaGraphLaunch(exec, s) == cudaSuccess;
            if (ok) ok = cudaStreamSynchronize(s) == cudaSuccess;
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            graphed = ok;
            g_last_graphed = ok ? 1 : 0;
            if (!ok) {
                cudaError_t e = cudaGetLastError();  // clear a non-sticky error
                (void)e;
            }
        }
        if (!graphed) {
            // same body replayed from the host, checking every 2 iterations
            BCtl hc;
            int it = 0;
            for (;;) {
                for (int t = 0; t < 2 && it < max_iters; ++t, ++it)
                    if ((st = launch_iteration(ws, plan, s, 0, 0)) != TV_OK) return st;
                st = check_cuda(cudaMemcpyAsync(&hc, ws.ctl, sizeof(hc), cudaMemcpyDeviceToHost, s),
                                "read control");
                if (st == TV_OK) st = check_cuda(cudaStreamSynchronize(s), "synchronize");
                if (st != TV_OK) return st;
                if (hc.active == 0 || it >= max_iters) break;
            }
        }
    }
    std::vector<BState> hs(n_imgs);
    st = check_cuda(cudaMemcpyAsync(hs.data(), ws.st, sizeof(BState) * n_imgs,
                                    cudaMemcpyDeviceToHost, s), "read states");
    if (st == TV_OK) st = check_cuda(cudaStreamSynchronize(s), "synchronize");
    if (st != TV_OK) return st;
    bool all = true;
    long long kernels = 0;
    for (int m = 0; m < n_imgs; ++m) {
        if (hs[m].k & 1) {
            st = check_cuda(cudaMemcpyAsync(imgs[m].x, plan.imgs[m].x1,
                                            sizeof(float) * (size_t)(imgs[m].H * imgs[m].W),
                                            cudaMemcpyDeviceToDevice, s), "copy x");
            if (st != TV_OK) return st;
        }
        if (iters_out) iters_out[m] = hs[m].k;
        if (gap_out) gap_out[m] = hs[m].gap;
        all = all && hs[m].done == 1;
        kernels = std::max(kernels, (long long)hs[m].k);
    }
    for (int m = 0; m < n_imgs; ++m) {
        if (!imgs[m].y_out) continue;
        st = check_cuda(cudaMemcpyAsync(imgs[m].y_out, plan.imgs[m].y,
                                        sizeof(float) * (size_t)(imgs[m].H * imgs[m].W),
                                        cudaMemcpyDeviceToDevice, s), "copy y");
        if (st != TV_OK) return st;
    }
    for (long long q = 0; q < 3 * kernels; ++q) note_launch();  // column, row, gap per iteration
    st = check_cuda(cudaStreamSynchronize(s), "synchronize");
    if (st != TV_OK) return st;
    return all ? TV_OK : TV_ERR_NOT_CONVERGED;
}

}  // extern "C"
