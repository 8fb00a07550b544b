// ROF denoising by the symmetric Lagrangian split of Sec. 6: the image is copied into
// a horizontal part x_h and a vertical part x_v, each carrying half of the data term,
// coupled by a multiplier y:
//     min_{x_h, x_v} max_y  Psi_h(x_h) + Psi_v(x_v) + <x_h - x_v, y>,
//     Psi_{h,v}(x) = TV_{h,v}(x) + 1/4 ||x - f||^2,
// solved by the primal-dual iteration printed in Sec. 6 for this split:
//     x_h <- prox_{tau_k Psi_h}(x_h - tau_k ybar)     (row chains)
//     x_v <- prox_{tau_k Psi_v}(x_v + tau_k ybar)     (column chains)
//     y_new = y + sigma_k (x_h - x_v),  ybar = y_new + theta (y_new - y),  y = y_new
// with tau_k = tau_0 / k, sigma_k = 1 / (tau_k L^2), L^2 = 2, theta = 1. Each proximal
// map is a batch of chain problems with curvature a = 1/2 + 1/tau_k, so the chains are
// solved with c = (f/2 + z/tau_k) / a and weights w / a by the warp-per-chain kernel.
// Stopping gap: P(xbar) - D(y), xbar = (x_h + x_v)/2, with the Lagrangian dual
//     D(y) = min_x [TV_h(x) + 1/4 ||x - f||^2 + <x, y>] + min_x [TV_v(x) + 1/4 ||x - f||^2 - <x, y>],
// a lower bound of the ROF minimum; each minimum is one chain batch (target f -+ 2y,
// weights 2w), evaluated every check_every iterations.
#include <cuda_runtime.h>

#include "tv_launch.cuh"

using namespace tvk;
using namespace tvh;

namespace {

// Row chains. MODE 0: the proximal step of x_h (in place); MODE 1: the row half of
// D(y) (c = f - 2y, weights 2w) into xout.
template <bool HAS_W, int MODE>
struct LagRowsP {
    static constexpr bool CREC = false;
    static constexpr bool UNIFORM_W = !HAS_W;  // one weight (a scaled lambda) per chain
    struct Raw {
        float f, x, y, w;
    };
    struct Acc {};
    const float *f, *x, *y, *wh;
    float *xout;
    float lam;
    long long H, W;
    float inv_tau, inv_a;

    __device__ bool resolve() { return true; }
    __device__ long long num_chains() const { return H; }
    __device__ int max_len() const { return (int)W; }
    __device__ bool chain(long long k, long long &start, int &n) const
    {
        start = k * W;
        n = (int)W;
        return true;
    }
    __device__ void fetch(long long k, long long start, int n, int i, Raw &r) const
    {
        const bool in = i < n;
        r.f = in ? f[start + i] : 0.f;
        r.x = (MODE == 0 && in) ? x[start + i] : 0.f;
        r.y = in ? y[start + i] : 0.f;
        r.w = (HAS_W && i < n - 1) ? wh[k * (W - 1) + i] : lam;
    }
    __device__ __forceinline__ void vals(float fv, float xv, float yv, float wv, float &c,
                                         float &w) const
    {
        if (MODE == 0) {
            c = (0.5f * fv + xv * inv_tau - yv) * inv_a;  // z = x_h - tau ybar
            w = wv * inv_a;
        } else {
            c = fv - 2.f * yv;
            w = 2.f * wv;
        }
    }
    __device__ void unary(long long, long long, int, int, const Raw &r, float &c, float &w,
                          Acc &) const
    {
        vals(r.f, r.x, r.y, r.w, c, w);
    }
    __device__ void unary_direct(int i, int n, long long k, long long start, float &c,
                                 float &w) const
    {
        Raw r;
        fetch(k, start, n, i, r);
        vals(r.f, r.x, r.y, r.w, c, w);
        if (i == n - 1) w = 0.f;
    }
    __device__ void emit(long long, long long start, int i, float xv, float) const
    {
        xout[start + i] = xv;
    }
    __device__ void emit_direct(int i, long long, long long start, float xv, float) const
    {
        xout[start + i] = xv;
    }
    __device__ long long spill_off(long long k, long long) const { return k * (2 * W + 2); }
    __device__ void acc_init(Acc &) const {}
    __device__ void finish(Acc &, int) const {}
    __device__ void finish_empty() const {}
};

// Column chains. MODE 0: the proximal step of x_v (z = x_v + tau ybar, in place);
// MODE 1: the column half of D(y) (c = f + 2y, weights 2w) into xout.
template <bool HAS_W, int MODE>
struct LagColsP {
    static constexpr bool CREC = false;
    static constexpr bool UNIFORM_W = !HAS_W;  // one weight (a scaled lambda) per chain
    struct Raw {
        float f, x, y, w;
    };
    struct Acc {};
    const float *f, *x, *y, *wv;
    float *xout;
    float lam;
    long long H, W;
    float inv_tau, inv_a;

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
        r.f = in ? f[o] : 0.f;
        r.x = (MODE == 0 && in) ? x[o] : 0.f;
        r.y = in ? y[o] : 0.f;
        r.w = (HAS_W && i < n - 1) ? wv[o] : lam;
    }
    __device__ __forceinline__ void vals(float fv, float xv, float yv, float wv, float &c,
                                         float &w) const
    {
        if (MODE == 0) {
            c = (0.5f * fv + xv * inv_tau + yv) * inv_a;  // z = x_v + tau ybar
            w = wv * inv_a;
        } else {
            c = fv + 2.f * yv;
            w = 2.f * wv;
        }
    }
    __device__ void unary(long long, long long, int, int, const Raw &r, float &c, float &w,
                          Acc &) const
    {
        vals(r.f, r.x, r.y, r.w, c, w);
    }
    __device__ void unary_direct(int i, int n, long long col, long long start, float &c,
                                 float &w) const
    {
        Raw r;
        fetch(col, start, n, i, r);
        vals(r.f, r.x, r.y, r.w, c, w);
        if (i == n - 1) w = 0.f;
    }
    __device__ void emit(long long col, long long, int i, float xv, float) const
    {
        xout[(long long)i * W + col] = xv;
    }
    __device__ void emit_direct(int i, long long col, long long, float xv, float) const
    {
        xout[(long long)i * W + col] = xv;
    }
    __device__ long long spill_off(long long col, long long) const { return col * (2 * H + 2); }
    __device__ void acc_init(Acc &) const {}
    __device__ void finish(Acc &, int) const {}
    __device__ void finish_empty() const {}
};

// Both proximal steps of one iteration in one launch: they read the same ybar (or y)
// and write separate iterates, so they are independent. Chains 0..H-1 are the rows,
// H..H+W-1 the columns (one warp per chain, so each warp takes one branch); the two
// latency-bound batches then share the GPU instead of running one after the other.
// Overflow reserves: the rows' first, then the columns'.
template <class PR, class PC>
struct LagBothP {
    static constexpr bool CREC = false;
    static_assert(!PR::CREC && !PC::CREC, "no c records");
    static constexpr bool UNIFORM_W = PR::UNIFORM_W && PC::UNIFORM_W;
    using Raw = typename PR::Raw;
    struct Acc {};
    PR r;
    PC c;

    __device__ bool resolve() { return r.resolve() && c.resolve(); }
    __device__ long long num_chains() const { return r.H + r.W; }
    __device__ int max_len() const { return (int)(r.H > r.W ? r.H : r.W); }
    __device__ bool chain(long long k, long long &start, int &n) const
    {
        return k < r.H ? r.chain(k, start, n) : c.chain(k - r.H, start, n);
    }
    __device__ void fetch(long long k, long long start, int n, int i, Raw &raw) const
    {
        if (k < r.H) {
            r.fetch(k, start, n, i, raw);
        } else {
            typename PC::Raw q;
            c.fetch(k - r.H, start, n, i, q);
            raw = Raw{q.f, q.x, q.y, q.w};
        }
    }
    __device__ void unary(long long k, long long start, int n, int i, const Raw &raw, float &cc,
                          float &w, Acc &) const
    {
        if (k < r.H) {
            typename PR::Acc a;
            r.unary(k, start, n, i, raw, cc, w, a);
        } else {
            typename PC::Acc a;
            c.unary(k - r.H, start, n, i, typename PC::Raw{raw.f, raw.x, raw.y, raw.w}, cc, w, a);
        }
    }
    __device__ void emit(long long k, long long start, int i, float xv, float cc) const
    {
        if (k < r.H) r.emit(k, start, i, xv, cc);
        else c.emit(k - r.H, start, i, xv, cc);
    }
    __device__ void unary_direct(int i, int n, long long k, long long start, float &cc,
                                 float &w) const
    {
        if (k < r.H) r.unary_direct(i, n, k, start, cc, w);
        else c.unary_direct(i, n, k - r.H, start, cc, w);
    }
    __device__ void emit_direct(int i, long long k, long long start, float xv, float cc) const
    {
        if (k < r.H) r.emit_direct(i, k, start, xv, cc);
        else c.emit_direct(i, k - r.H, start, xv, cc);
    }
    __device__ long long spill_off(long long k, long long start) const
    {
        return k < r.H ? r.spill_off(k, start) : r.H * (2 * r.W + 2) + c.spill_off(k - r.H, start);
    }
    __device__ void acc_init(Acc &) const {}
    __device__ void finish(Acc &, int) const {}
    __device__ void finish_empty() const {}
};

// y_new = y + sigma (x_h - x_v); ybar = 2 y_new - y; y = y_new; xbar = (x_h + x_v) / 2.
__global__ void lag_dual_update(long long N, const float *xh, const float *xv, float *y,
                                float *ybar, float *xbar, float sigma)
{
    pdl_enter();
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < N;
         q += (long long)gridDim.x * blockDim.x) {
        const float yo = y[q];
        const float yn = yo + sigma * (xh[q] - xv[q]);
        ybar[q] = yn + (yn - yo);
        y[q] = yn;
        xbar[q] = 0.5f * (xh[q] + xv[q]);
    }
}

constexpr int kLagThreads = 256;

// Per-pixel terms of P(xbar) - D(y); FP32 over at most 32 pixels per thread, FP64
// beyond; the last block sums the block partials in a fixed order into *gap (per pixel).
__global__ void __launch_bounds__(kLagThreads)
    lag_gap_kernel(const float *f, const float *wh, const float *wv, float lam, long long H,
                   long long W, const float *xbar, const float *xr, const float *xc,
                   const float *y, double *partials, unsigned *ticket, double *gap)
{
    __shared__ double red[kLagThreads];
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
        const float fv = f[q], xb = xbar[q], a = xr[q], b = xc[q], yv = y[q];
        float t = 0.5f * (xb - fv) * (xb - fv) - 0.25f * (a - fv) * (a - fv) - a * yv -
                  0.25f * (b - fv) * (b - fv) + b * yv;
        if (c + 1 < W) {
            const float wq = wh ? wh[r * (W - 1) + c] : lam;
            t += wq * (fabsf(xbar[q + 1] - xb) - fabsf(xr[q + 1] - a));
        }
        if (r + 1 < H) {
            const float wq = wv ? wv[q] : lam;
            t += wq * (fabsf(xbar[q + W] - xb) - fabsf(xc[q + W] - b));
        }
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
    for (int h = kLagThreads / 2; h > 0; h >>= 1) {
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
    for (int h = kLagThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *gap = red[0] / (double)N;
        *ticket = 0;
    }
}

struct LagWs {
    float *xh, *xv, *y, *ybar, *xr, *xc;
    float2 *rec, *spill;
    WsHeader *hdr;
    double *partials, *gap;
    unsigned *ticket;
    size_t bytes;
};

int lag_gap_blocks(long long N)
{
    long long b = (N + kLagThreads * 8 - 1) / (kLagThreads * 8);
    const long long cap = 4LL * sm_count_current();
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

LagWs carve_lag(void *base, long long H, long long W, int gap_blocks)
{
    Carver cv(base);
    LagWs o;
    const long long N = H * W;
    o.hdr = cv.take<WsHeader>(1);
    o.gap = cv.take<double>(1);
    o.ticket = cv.take<unsigned>(1);
    o.partials = cv.take<double>((size_t)gap_blocks);
    o.xh = cv.take<float>((size_t)N);
    o.xv = cv.take<float>((size_t)N);
    o.y = cv.take<float>((size_t)N);
    o.ybar = cv.take<float>((size_t)N);
    o.xr = cv.take<float>((size_t)N);
    o.xc = cv.take<float>((size_t)N);
    // records of the row and column chains of one launch (at chain * max(H, W)) and
    // their overflow reserves side by side
    o.rec = cv.take<float2>((size_t)((H + W) * std::max(H, W)));
    o.spill = cv.take<float2>((size_t)(H * (2 * W + 2) + W * (2 * H + 2)));
    o.bytes = align_up(cv.used, 256);
    return o;
}

template <int MODE, bool HW_, bool VW_>
tv_status lag_both_t(const float *f, const float *xh, const float *xv, const float *y,
                     const float *wh, const float *wv, float lam, long long H, long long W,
                     float *xout_h, float *xout_v, float inv_tau, float inv_a, const LagWs &ws,
                     cudaStream_t s)
{
    LagBothP<LagRowsP<HW_, MODE>, LagColsP<VW_, MODE>> p{
        {f, xh, y, wh, xout_h, lam, H, W, inv_tau, inv_a},
        {f, xv, y, wv, xout_v, lam, H, W, inv_tau, inv_a}};
    return launch_coop(p, H + W, (int)std::max(H, W), ws.rec, nullptr, ws.spill, ws.hdr, s,
                       PK_ROW);
}

// The row and the column chains of one iteration (MODE 0: the proximal steps of x_h and
// x_v; MODE 1: the two halves of D(y)) in one launch.
template <int MODE>
tv_status lag_both(const float *f, const float *xh, const float *xv, const float *y,
                   const float *wh, const float *wv, float lam, long long H, long long W,
                   float *xout_h, float *xout_v, float inv_tau, float inv_a, const LagWs &ws,
                   cudaStream_t s)
{
    if (wh && wv)
        return lag_both_t<MODE, true, true>(f, xh, xv, y, wh, wv, lam, H, W, xout_h, xout_v,
                                            inv_tau, inv_a, ws, s);
    if (wh)
        return lag_both_t<MODE, true, false>(f, xh, xv, y, wh, wv, lam, H, W, xout_h, xout_v,
                                             inv_tau, inv_a, ws, s);
    if (wv)
        return lag_both_t<MODE, false, true>(f, xh, xv, y, wh, wv, lam, H, W, xout_h, xout_v,
                                             inv_tau, inv_a, ws, s);
    return lag_both_t<MODE, false, false>(f, xh, xv, y, wh, wv, lam, H, W, xout_h, xout_v,
                                          inv_tau, inv_a, ws, s);
}

int ew_blocks(long long n) { return (int)std::min<long long>((n + 255) / 256, 8LL * sm_count_current()); }

}  // namespace

extern "C" {

size_t tv2d_lagrangian_workspace_size(int64_t H, int64_t W)
{
    if (H < 1 || W < 1) return 0;
    return carve_lag(nullptr, H, W, lag_gap_blocks(H * W)).bytes;
}

tv_status tv2d_denoise_lagrangian(const float *d_img, int64_t H, int64_t W, const float *d_wh,
                                  const float *d_wv, float lambda, float tau0, int max_iters,
                                  double gap_tol, int check_every, float *d_x, int *iters_out,
                                  double *gap_out, void *d_workspace, size_t workspace_bytes,
                                  tv_stream_t stream)
{
    clear_error();
    if (H < 1 || W < 1 || H > (1LL << 24) || W > (1LL << 24) || max_iters < 1 ||
        check_every < 1 || !(tau0 > 0.f && tau0 < INFINITY)) {
        set_error("tv2d_denoise_lagrangian: need H, W >= 1, max_iters >= 1, check_every >= 1 "
                  "and a finite tau0 > 0");
        return TV_ERR_INVALID;
    }
    if (!d_img || !d_x || !d_workspace) {
        set_error("tv2d_denoise_lagrangian: img, x and workspace must not be NULL");
        return TV_ERR_INVALID;
    }
    if (!(gap_tol >= 0.0 && gap_tol < INFINITY)) {
        set_error("tv2d_denoise_lagrangian: gap_tol must be finite and >= 0");
        return TV_ERR_INVALID;
    }
    if ((!d_wh || !d_wv) && !(lambda >= 0.f && lambda < INFINITY)) {
        set_error("tv2d_denoise_lagrangian: lambda must be finite and >= 0");
        return TV_ERR_INVALID;
    }
    const long long N = H * W;
    const size_t npx = (size_t)N * sizeof(float);
    const int gb = lag_gap_blocks(N);
    LagWs ws = carve_lag(d_workspace, H, W, gb);
    if (workspace_bytes < ws.bytes) {
        set_error("tv2d_denoise_lagrangian: workspace of %zu bytes, %zu needed", workspace_bytes,
                  ws.bytes);
        return TV_ERR_NOMEM;
    }
    {
        const char *a = (const char *)d_x, *b = (const char *)d_img;
        if (a < b + npx && b < a + npx) {
            set_error("tv2d_denoise_lagrangian: x must not overlap the image");
            return TV_ERR_INVALID;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    tv_status st;
    if ((st = check_cuda(cudaMemsetAsync(ws.hdr, 0, sizeof(WsHeader), s), "memset")) != TV_OK ||
        (st = check_cuda(cudaMemsetAsync(ws.ticket, 0, sizeof(unsigned), s), "memset")) != TV_OK ||
        (st = check_cuda(cudaMemcpyAsync(ws.xh, d_img, npx, cudaMemcpyDeviceToDevice, s), "copy")) !=
            TV_OK ||
        (st = check_cuda(cudaMemcpyAsync(ws.xv, d_img, npx, cudaMemcpyDeviceToDevice, s), "copy")) !=
            TV_OK ||
        (st = check_cuda(cudaMemsetAsync(ws.y, 0, npx, s), "memset")) != TV_OK ||
        (st = check_cuda(cudaMemsetAsync(ws.ybar, 0, npx, s), "memset")) != TV_OK)
        return st;
    double gap = NAN;
    int k = 1;
    bool done = false;
    PdlScope pdl(true);  // each kernel may become resident while its predecessor finishes
    for (; k <= max_iters; ++k) {
        const double tau = (double)tau0 / k;
        const float inv_tau = (float)(1.0 / tau), inv_a = (float)(1.0 / (0.5 + 1.0 / tau));
        const float sigma = (float)(1.0 / (2.0 * tau));
        // the proximal steps of x_h (rows) and x_v (columns), in place, in one launch
        if ((st = lag_both<0>(d_img, ws.xh, ws.xv, ws.ybar, d_wh, d_wv, lambda, H, W, ws.xh, ws.xv,
                              inv_tau, inv_a, ws, s)) != TV_OK)
            return st;
        if ((st = check_cuda(launch_k(lag_dual_update, dim3(ew_blocks(N)), dim3(256), 0, s, N,
                                      (const float *)ws.xh, (const float *)ws.xv, ws.y, ws.ybar,
                                      d_x, sigma),
                             "dual update")) != TV_OK)
            return st;
        note_launch();
        if (k % check_every == 0 || k == max_iters) {
            // the two halves of D(y) (rows into xr, columns into xc) in one launch
            if ((st = lag_both<1>(d_img, nullptr, nullptr, ws.y, d_wh, d_wv, lambda, H, W, ws.xr,
                                  ws.xc, 0.f, 0.f, ws, s)) != TV_OK)
                return st;
            if ((st = check_cuda(launch_k(lag_gap_kernel, dim3(gb), dim3(kLagThreads), 0, s, d_img,
                                          d_wh, d_wv, lambda, H, W, (const float *)d_x,
                                          (const float *)ws.xr, (const float *)ws.xc,
                                          (const float *)ws.y, ws.partials, ws.ticket, ws.gap),
                                 "gap")) != TV_OK)
                return st;
            note_launch();
            st = check_cuda(cudaMemcpyAsync(&gap, ws.gap, sizeof(double), cudaMemcpyDeviceToHost, s),
                            "read gap");
            if (st == TV_OK) st = check_cuda(cudaStreamSynchronize(s), "synchronize");
            if (st != TV_OK) return st;
            if (gap_tol > 0.0 && gap <= gap_tol) {
                done = true;
                break;
            }
        }
    }
    if (iters_out) *iters_out = done ? k : max_iters;
    if (gap_out) *gap_out = gap;
    return done ? TV_OK : TV_ERR_NOT_CONVERGED;
}

}  // extern "C"
