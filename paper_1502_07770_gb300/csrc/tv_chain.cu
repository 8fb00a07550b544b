// Batched chain TV-l2 solves (eq. 1D-ROF) behind the C ABI: contiguous chains
// given by CSR offsets (or a uniform length), and the column chains of a
// row-major array. One thread per chain runs the dynamic program of Algorithm 2
// / Sec. 4.1 (tv_dp.cuh).
#include <cuda_runtime.h>

#include <atomic>
#include <array>
#include <mutex>
#include <vector>

#include "tv_flat.cuh"
#include "tv_halves.cuh"
#include "tv_launch.cuh"

namespace tvh {

static thread_local char g_err[512];

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

tv_status check_cuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return TV_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return TV_ERR_CUDA;
}

int sm_count_current()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
    return sms > 0 ? sms : 148;
}

// ---------------------------------------------------------- launch accounting --
static std::atomic<long long> g_launches{0};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
struct ProfPair {
    cudaEvent_t a, b;
};
static std::vector<ProfPair> g_prof_pending[PK_N];
static std::vector<ProfPair> g_prof_free;
static cudaEvent_t g_prof_open[PK_N];
static double g_prof_ms[PK_N];
static long long g_prof_n[PK_N];

void note_launch() { g_launches.fetch_add(1); }

static std::atomic<long long> g_coop_max{kCoopMaxChainsDefault};
static std::atomic<bool> g_coop_auto{true};
long long coop_max_chains() { return g_coop_max.load(); }
bool coop_max_auto() { return g_coop_auto.load(); }
static std::atomic<int> g_coop_split{1};
int coop_split() { return g_coop_split.load(); }
static std::atomic<int> g_thread_split{2};
int thread_split() { return g_thread_split.load(); }

// programmatic dependent launch: enabled by the ABI switch, active inside a PdlScope
static std::atomic<int> g_pdl_enabled{1};
static thread_local bool g_pdl_scope = false;
bool pdl_on() { return g_pdl_scope; }
PdlScope::PdlScope(bool on) : prev(g_pdl_scope) { g_pdl_scope = on && g_pdl_enabled.load() != 0; }
PdlScope::~PdlScope() { g_pdl_scope = prev; }
bool prof_on() { return g_prof_on; }

void prof_mark(int kind, cudaStream_t s, bool start)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (start) {
        ProfPair pr;
        if (!g_prof_free.empty()) {
            pr = g_prof_free.back();
            g_prof_free.pop_back();
        } else {
            cudaEventCreate(&pr.a);
            cudaEventCreate(&pr.b);
        }
        cudaEventRecord(pr.a, s);
        g_prof_open[kind] = pr.b;
        g_prof_pending[kind].push_back(pr);
    } else if (!g_prof_pending[kind].empty()) {
        cudaEventRecord(g_prof_pending[kind].back().b, s);
    }
}

size_t prof_pending(int kind)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    return g_prof_pending[kind].size();
}

void prof_drop_from(int kind, size_t first)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::vector<ProfPair> &v = g_prof_pending[kind];
    while (v.size() > first) {
        cudaEventSynchronize(v.back().b);
        g_prof_free.push_back(v.back());
        v.pop_back();
    }
}

static void prof_collect(int kind)
{
    for (ProfPair &pr : g_prof_pending[kind]) {
        float ms = 0.f;
        cudaEventSynchronize(pr.b);
        if (cudaEventElapsedTime(&ms, pr.a, pr.b) == cudaSuccess) {
            g_prof_ms[kind] += ms;
            g_prof_n[kind] += 1;
        }
        g_prof_free.push_back(pr);
    }
    g_prof_pending[kind].clear();
}

Shape batch_shape(long long warps, int sm_count)
{
    // Spread small batches over many SMs (the DP is latency-bound); group large
    // batches four warps per block so that two blocks share an SM.
    int wpb = (int)(warps / (2LL * sm_count));
    if (wpb < 1) wpb = 1;
    if (wpb > 4) wpb = 4;
    return Shape{wpb, (warps + wpb - 1) / wpb};
}

Shape chains_shape(long long warps, const void *kern, size_t per_warp)
{
    const int sms = sm_count_current();
    if (warps < 2LL * sms) return batch_shape(warps, sms);
    static std::mutex mu;
    static std::vector<std::pair<const void *, std::array<int, 5>>> cache;
    std::array<int, 5> per_sm{};  // resident blocks per SM for 1..4 warps per block
    {
        std::lock_guard<std::mutex> lk(mu);
        bool found = false;
        for (auto &e : cache)
            if (e.first == kern) {
                per_sm = e.second;
                found = true;
            }
        if (!found) {
            for (int w = 1; w <= 4; ++w) {
                int b = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, w * tvk::WARP, w * per_warp) !=
                    cudaSuccess) {
                    (void)cudaGetLastError();
                    b = 0;
                }
                per_sm[w] = b;
            }
            cache.push_back({kern, per_sm});
        }
    }
    int best = 0;
    long long best_res = -1;
    for (int w = 4; w >= 1; --w) {
        const long long res = (long long)per_sm[w] * w * sms;
        if (res >= warps) return Shape{w, (warps + w - 1) / w};
        if (res > best_res) {
            best_res = res;
            best = w;
        }
    }
    if (best == 0 || best_res <= 0) return batch_shape(warps, sms);
    return Shape{best, (warps + best - 1) / best};
}

}  // namespace tvh

using namespace tvk;
using namespace tvh;

namespace {

constexpr int kRing = 32;

// CSR batches: the node range [offsets[0], offsets[num_chains]) of x must not overlap
// that of y or of w (the host checks only x == y, since the offsets live on the device).
// Read by every thread at kernel entry; an overlap flags ERR_BAD_CHAIN and skips the
// whole launch.
__device__ __forceinline__ bool csr_disjoint(const float *x, const float *y, const float *w,
                                             long long off0, long long offn)
{
    if (offn <= off0) return true;
    const size_t len = (size_t)(offn - off0) * sizeof(float);
    auto apart = [&](const float *a) {
        if (a == nullptr) return true;
        const uintptr_t p = (uintptr_t)(x + off0), q = (uintptr_t)(a + off0);
        return p + len <= q || q + len <= p;
    };
    return apart(y) && apart(w);
}

// Contiguous chains: chain k at [off_k, off_{k+1}) (or [k*len, (k+1)*len)).
template <bool HAS_W>
struct ChainRowsP {
    static constexpr bool COLS = false;
    static constexpr int NIN = HAS_W ? 2 : 1;
    static constexpr int WI = HAS_W ? 1 : -1;  // the weights input
    static constexpr bool NEIGH = false;
    static constexpr bool CREC = false;
    static constexpr int NOUT = 1;
    struct Acc {};

    const float *y, *w;
    float lam;
    const int64_t *offsets;
    long long nchains;
    int maxlen;
    float *x;
    bool vec;        // uniform chains, length % 4 == 0, 16-byte aligned arrays
    long long off0;  // offsets[0], so that reserve slices start at zero
    int *status;     // workspace error word (CSR overlap check), or NULL

    __device__ bool resolve()
    {
        off0 = offsets ? (long long)offsets[0] : 0;
        if (offsets && !csr_disjoint(x, y, w, off0, (long long)offsets[nchains])) {
            if (status && threadIdx.x == 0) atomicOr(status, ERR_BAD_CHAIN);
            return false;
        }
        return true;
    }
    __device__ long long num_chains() const { return nchains; }
    __device__ int max_len() const { return maxlen; }
    __device__ bool chain(long long k, long long &start, int &n) const
    {
        if (offsets) {
            const long long a = offsets[k], b = offsets[k + 1];
            // monotone offsets keep every chain inside the first (k+1)*max_len nodes
            // after offsets[0]; that also bounds its slice of the reserve
            if (a < off0 || b < a || b - a > maxlen || b - off0 > (k + 1) * (long long)maxlen)
                return false;
            start = a;
            n = (int)(b - a);
        } else {
            start = k * (long long)maxlen;
            n = maxlen;
        }
        return true;
    }
    __device__ const float *in_ptr(int a) const { return a == 0 ? y : w; }
    __device__ long long in_off(int, long long, long long start) const { return start; }
    __device__ int in_lim(int a, int n) const { return a == 0 ? n : n - 1; }
    __device__ long long in_ld(int) const { return 1; }
    __device__ long long in_kmax(int) const { return nchains; }
    __device__ bool in_vec(int) const { return vec; }
    __device__ bool out_vec() const { return vec; }
    __device__ void unary(const float (&v)[NIN], float, int, int i, int n, long long, float &c,
                          float &wi, Acc &) const
    {
        c = v[0];
        if constexpr (HAS_W) wi = (i < n - 1) ? v[NIN - 1] : 0.f;
        else wi = (i < n - 1) ? lam : 0.f;
    }
    __device__ void unary_direct(int i, int n, long long, long long start, float &c,
                                 float &wi) const
    {
        c = y[start + i];
        if constexpr (HAS_W) wi = (i < n - 1) ? w[start + i] : 0.f;
        else wi = (i < n - 1) ? lam : 0.f;
    }
    __device__ float *out_ptr(int) const { return x; }
    __device__ long long out_off(int, long long, long long start) const { return start; }
    __device__ void emit_cols(int, long long, float, float) const {}
    __device__ void emit_direct(int i, long long, long long start, float xv, float) const
    {
        x[start + i] = xv;
    }
    __device__ long long spill_off(long long k, long long start) const
    {
        return 2 * (start - off0) + 2 * k;  // 2n+2 entries per chain
    }
    __device__ void acc_init(Acc &) const {}
    __device__ void finish(Acc &) const {}
    __device__ void finish_empty() const {}
};

// Column chains of an H x W array with leading dimension ld.
template <bool HAS_W>
struct ChainColsP {
    static constexpr bool COLS = true;
    static constexpr int NIN = HAS_W ? 2 : 1;
    static constexpr bool NEIGH = false;
    static constexpr bool CREC = false;
    static constexpr int NOUT = 0;
    struct Acc {};

    const float *y, *w;
    float lam;
    long long H, W, ld;
    float *x;
    bool vec;  // ld % 4 == 0 and 16-byte aligned arrays

    __device__ bool resolve() { return true; }
    __device__ long long num_chains() const { return W; }
    __device__ int max_len() const { return (int)H; }
    __device__ bool chain(long long k, long long &start, int &n) const
    {
        start = k;
        n = (int)H;
        return true;
    }
    __device__ const float *in_ptr(int a) const { return a == 0 ? y : w; }
    __device__ long long in_off(int, long long, long long start) const { return start; }
    __device__ int in_lim(int a, int n) const { return a == 0 ? n : n - 1; }
    __device__ long long in_ld(int) const { return ld; }
    __device__ long long in_kmax(int) const { return W; }
    __device__ bool in_vec(int) const { return vec; }
    __device__ bool out_vec() const { return vec; }
    __device__ void unary(const float (&v)[NIN], float, int, int i, int n, long long, float &c,
                          float &wi, Acc &) const
    {
        c = v[0];
        if constexpr (HAS_W) wi = (i < n - 1) ? v[NIN - 1] : 0.f;
        else wi = (i < n - 1) ? lam : 0.f;
    }
    __device__ void unary_direct(int i, int n, long long k, long long, float &c, float &wi) const
    {
        c = y[(long long)i * ld + k];
        if constexpr (HAS_W) wi = (i < n - 1) ? w[(long long)i * ld + k] : 0.f;
        else wi = (i < n - 1) ? lam : 0.f;
    }
    __device__ float *out_ptr(int) const { return x; }
    __device__ long long out_off(int, long long, long long) const { return 0; }
    __device__ void emit_cols(int i, long long k, float xv, float) const
    {
        if (k < W) x[(long long)i * ld + k] = xv;
    }
    __device__ void emit_direct(int i, long long k, long long, float xv, float) const
    {
        x[(long long)i * ld + k] = xv;
    }
    __device__ long long spill_off(long long k, long long) const { return k * (2 * H + 2); }
    __device__ void acc_init(Acc &) const {}
    __device__ void finish(Acc &) const {}
    __device__ void finish_empty() const {}
};

// ---- the same batches, one warp per chain (tv_coop.cuh) ----
template <bool HAS_W>
struct CoopRowsP {
    static constexpr bool CREC = false;
    static constexpr bool UNIFORM_W = !HAS_W;  // one weight (a scaled lambda) per chain
    struct Raw {
        float y, w;
    };
    struct Acc {};

    const float *y, *w;
    float lam;
    const int64_t *offsets;
    long long nchains;
    int maxlen;
    float *x;
    long long off0;
    int *status;  // workspace error word (CSR overlap check), or NULL

    __device__ bool resolve()
    {
        off0 = offsets ? (long long)offsets[0] : 0;
        if (offsets && !csr_disjoint(x, y, w, off0, (long long)offsets[nchains])) {
            if (status && threadIdx.x == 0) atomicOr(status, ERR_BAD_CHAIN);
            return false;
        }
        return true;
    }
    __device__ long long num_chains() const { return nchains; }
    __device__ int max_len() const { return maxlen; }
    __device__ bool chain(long long k, long long &start, int &n) const
    {
        if (offsets) {
            const long long a = offsets[k], b = offsets[k + 1];
            if (a < off0 || b < a || b - a > maxlen || b - off0 > (k + 1) * (long long)maxlen)
                return false;
            start = a;
            n = (int)(b - a);
        } else {
            start = k * (long long)maxlen;
            n = maxlen;
        }
        return true;
    }
    __device__ void fetch(long long, long long start, int n, int i, Raw &r) const
    {
        r.y = (i < n) ? y[start + i] : 0.f;
        if constexpr (HAS_W) r.w = (i < n - 1) ? w[start + i] : 0.f;
    }
    __device__ void unary(long long, long long, int, int, const Raw &r, float &c, float &wi,
                          Acc &) const
    {
        c = r.y;
        if constexpr (HAS_W) wi = r.w;
        else wi = lam;
    }
    __device__ void emit(long long, long long start, int i, float xv, float) const
    {
        x[start + i] = xv;
    }
    __device__ void unary_direct(int i, int n, long long, long long start, float &c,
                                 float &wi) const
    {
        c = y[start + i];
        if constexpr (HAS_W) wi = (i < n - 1) ? w[start + i] : 0.f;
        else wi = (i < n - 1) ? lam : 0.f;
    }
    __device__ void emit_direct(int i, long long, long long start, float xv, float) const
    {
        x[start + i] = xv;
    }
    __device__ long long spill_off(long long k, long long start) const
    {
        return 2 * (start - off0) + 2 * k;
    }
    __device__ void acc_init(Acc &) const {}
    __device__ void finish(Acc &, int) const {}
    __device__ void finish_empty() const {}
};

template <bool HAS_W>
struct CoopColsP {
    static constexpr bool CREC = false;
    static constexpr bool UNIFORM_W = !HAS_W;  // one weight (a scaled lambda) per chain
    struct Raw {
        float y, w;
    };
    struct Acc {};

    const float *y, *w;
    float lam;
    long long H, W, ld;
    float *x;

    __device__ bool resolve() { return true; }
    __device__ long long num_chains() const { return W; }
    __device__ int max_len() const { return (int)H; }
    __device__ bool chain(long long k, long long &start, int &n) const
    {
        start = k;
        n = (int)H;
        return true;
    }
    __device__ void fetch(long long k, long long, int n, int i, Raw &r) const
    {
        r.y = (i < n) ? y[(long long)i * ld + k] : 0.f;
        if constexpr (HAS_W) r.w = (i < n - 1) ? w[(long long)i * ld + k] : 0.f;
    }
    __device__ void unary(long long, long long, int, int, const Raw &r, float &c, float &wi,
                          Acc &) const
    {
        c = r.y;
        if constexpr (HAS_W) wi = r.w;
        else wi = lam;
    }
    __device__ void emit(long long k, long long, int i, float xv, float) const
    {
        x[(long long)i * ld + k] = xv;
    }
    __device__ void unary_direct(int i, int n, long long k, long long, float &c, float &wi) const
    {
        c = y[(long long)i * ld + k];
        if constexpr (HAS_W) wi = (i < n - 1) ? w[(long long)i * ld + k] : 0.f;
        else wi = (i < n - 1) ? lam : 0.f;
    }
    __device__ void emit_direct(int i, long long k, long long, float xv, float) const
    {
        x[(long long)i * ld + k] = xv;
    }
    __device__ long long spill_off(long long k, long long) const { return k * (2 * H + 2); }
    __device__ void acc_init(Acc &) const {}
    __device__ void finish(Acc &, int) const {}
    __device__ void finish_empty() const {}
};

// ---- general convex chains (Sec. 4, Sec. 4.1), one warp per chain ----
struct GenRowsP {
    static constexpr bool CREC = false;
    struct Raw {
        float a, b, wl, wh;
    };
    struct Acc {};

    const float *a, *b, *wlo, *whi;
    const int64_t *offsets;
    long long nchains;
    int maxlen;
    float *x;
    long long off0;

    __device__ bool resolve()
    {
        off0 = offsets ? (long long)offsets[0] : 0;
        return true;
    }
    __device__ long long num_chains() const { return nchains; }
    __device__ int max_len() const { return maxlen; }
    __device__ bool chain(long long k, long long &start, int &n) const
    {
        if (offsets) {
            const long long lo = offsets[k], hi = offsets[k + 1];
            if (lo < off0 || hi < lo || hi - lo > maxlen || hi - off0 > (k + 1) * (long long)maxlen)
                return false;
            start = lo;
            n = (int)(hi - lo);
        } else {
            start = k * (long long)maxlen;
            n = maxlen;
        }
        return true;
    }
    __device__ void fetch(long long, long long start, int n, int i, Raw &r) const
    {
        const bool in = i < n, e = i < n - 1;
        r.a = in ? (a ? a[start + i] : 1.f) : 1.f;
        r.b = in ? b[start + i] : 0.f;
        r.wl = e ? wlo[start + i] : 0.f;
        r.wh = e ? whi[start + i] : 0.f;
    }
    __device__ void unary_g(long long, long long, int, int, const Raw &r, float &ai, float &bi,
                            float &wl, float &wh, Acc &) const
    {
        ai = r.a;
        bi = r.b;
        wl = r.wl;
        wh = r.wh;
    }
    __device__ void unary_g_direct(int i, int n, long long, long long start, float &ai, float &bi,
                                   float &wl, float &wh) const
    {
        ai = a ? a[start + i] : 1.f;
        bi = b[start + i];
        wl = (i < n - 1) ? wlo[start + i] : 0.f;
        wh = (i < n - 1) ? whi[start + i] : 0.f;
    }
    __device__ void emit(long long, long long start, int i, float xv, float) const
    {
        x[start + i] = xv;
    }
    __device__ long long spill_off(long long k, long long start) const
    {
        return 2 * (start - off0) + 2 * k;
    }
    __device__ void acc_init(Acc &) const {}
    __device__ void finish(Acc &, int) const {}
    __device__ void finish_empty() const {}
};

template <class P>
tv_status launch_batch(const P &p, long long nchains, float2 *rec, float *crec, float2 *spill,
                       WsHeader *hdr, cudaStream_t s)
{
    return launch_chains<P, kRing>(p, nchains, rec, crec, spill, hdr, s, PK_CHAIN);
}

// ----------------------------------------------- middle-rooted thread chains --
// tv_halves.cuh: one thread per chain half. A 16-entry ring per half keeps every warp
// of a full batch resident (27 per SM at 65536 chains); longer messages take the
// workspace path.
constexpr int kRingHalf = 16;

constexpr int kHalvesMinLen = 64;
constexpr int kFlatMinLenW = 1024;

template <bool HAS_W>
tv_status launch_halves(const ChainRowsP<HAS_W> &p, long long nchains, int max_len, float2 *rec,
                        float2 *spill, WsHeader *hdr, cudaStream_t s)
{
    const long long warps = (nchains + HW - 1) / HW;
    const size_t per_warp = sizeof(HalfSmem<ChainRowsP<HAS_W>, kRingHalf>);
    auto kern = chain_halves_kernel<ChainRowsP<HAS_W>, kRingHalf>;
    tv_status st = check_cuda(
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(4 * per_warp)),
        "cudaFuncSetAttribute");
    if (st != TV_OK) return st;
    const Shape sh = chains_shape(warps, (const void *)kern, per_warp);
    const bool prof = prof_on();
    if (prof) prof_mark(PK_CHAIN, s, true);
    kern<<<(unsigned)sh.blocks, sh.wpb * WARP, sh.wpb * per_warp, s>>>(p, rec, nullptr, spill, hdr,
                                                                       (max_len + 1) / 2);
    st = check_cuda(cudaGetLastError(), "chain halves kernel launch");
    if (st == TV_OK) note_launch();
    if (prof) prof_mark(PK_CHAIN, s, false);
    return st;
}

// chain_flat_kernel (tv_flat.cuh): one thread per chain half, fixed-shape update.
template <bool HAS_W>
tv_status launch_flat(const ChainRowsP<HAS_W> &p, long long nchains, int max_len, float2 *rec,
                      float2 *spill, WsHeader *hdr, cudaStream_t s)
{
    const long long warps = (nchains + HW - 1) / HW;
    const size_t per_warp = sizeof(FlatSmem<HAS_W ? 2 : 1>);
    auto kern = p.vec ? chain_flat_kernel<ChainRowsP<HAS_W>, true> : chain_flat_kernel<ChainRowsP<HAS_W>, false>;
    tv_status st = check_cuda(
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(4 * per_warp)),
        "cudaFuncSetAttribute");
    if (st != TV_OK) return st;
    const Shape sh = chains_shape(warps, (const void *)kern, per_warp);
    const bool prof = prof_on();
    if (prof) prof_mark(PK_CHAIN, s, true);
    kern<<<(unsigned)sh.blocks, sh.wpb * WARP, sh.wpb * per_warp, s>>>(p, rec, spill, hdr,
                                                                       (max_len + 1) / 2);
    st = check_cuda(cudaGetLastError(), "chain flat kernel launch");
    if (st == TV_OK) note_launch();
    if (prof) prof_mark(PK_CHAIN, s, false);
    return st;
}

struct ChainWs {
    WsHeader *hdr;
    float2 *rec;
    float2 *spill;
    size_t bytes;
};

ChainWs carve_chain_ws(void *ws, long long warps, long long max_len, long long spill_entries)
{
    Carver cv(ws);
    ChainWs o;
    o.hdr = cv.take<WsHeader>(1);
    o.rec = cv.take<float2>((size_t)(warps * max_len * WARP));
    o.spill = cv.take<float2>((size_t)spill_entries);
    o.bytes = align_up(cv.used, 256);
    return o;
}

// 16-byte copies need every array 16-byte aligned and rows of a multiple of 4 floats.
bool vec_ok(const int64_t *offsets, long long row, const void *a, const void *b, const void *c)
{
    auto al = [](const void *q) { return q == nullptr || ((uintptr_t)q & 15) == 0; };
    return offsets == nullptr && row % 4 == 0 && al(a) && al(b) && al(c);
}

bool overlaps(const void *a, size_t an, const void *b, size_t bn)
{
    if (!a || !b || an == 0 || bn == 0) return false;
    const char *pa = (const char *)a, *pb = (const char *)b;
    return pa < pb + bn && pb < pa + an;
}

}  // namespace

extern "C" {

const char *tv_last_error(void) { return tvh::g_err; }

int tv_version(void) { return 100; }

int64_t tv_launch_count(void) { return (int64_t)tvh::g_launches.load(); }

tv_status tv_set_coop_max_chains(int64_t max_chains)
{
    clear_error();
    if (max_chains < 0) {
        set_error("tv_set_coop_max_chains: must be >= 0");
        return TV_ERR_INVALID;
    }
    tvh::g_coop_max.store(max_chains == 0 ? kCoopMaxChainsDefault : max_chains);
    tvh::g_coop_auto.store(max_chains == 0);
    return TV_OK;
}

tv_status tv_set_programmatic_launch(int on)
{
    clear_error();
    if (on < 0 || on > 1) {
        set_error("tv_set_programmatic_launch: 0 or 1");
        return TV_ERR_INVALID;
    }
    tvh::g_pdl_enabled.store(on);
    return TV_OK;
}

tv_status tv_set_thread_split(int on)
{
    clear_error();
    if (on < 0 || on > 2) {
        set_error("tv_set_thread_split: 0, 1 or 2");
        return TV_ERR_INVALID;
    }
    tvh::g_thread_split.store(on);
    return TV_OK;
}

tv_status tv_set_coop_split(int on)
{
    clear_error();
    if (on < 0 || on > 2) {
        set_error("tv_set_coop_split: 0, 1 or 2");
        return TV_ERR_INVALID;
    }
    tvh::g_coop_split.store(on);
    return TV_OK;
}

tv_status tv_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(tvh::g_prof_mu);
    tvh::g_prof_on = on != 0;
    return TV_OK;
}

tv_status tv_profile_read(int kind, double *total_ms, int64_t *launches)
{
    clear_error();
    if (kind < 0 || kind >= PK_N || !total_ms || !launches) {
        set_error("tv_profile_read: kind must be 0..4 and the outputs non-NULL");
        return TV_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(tvh::g_prof_mu);
    tvh::prof_collect(kind);
    *total_ms = tvh::g_prof_ms[kind];
    *launches = (int64_t)tvh::g_prof_n[kind];
    tvh::g_prof_ms[kind] = 0.0;
    tvh::g_prof_n[kind] = 0;
    return TV_OK;
}

size_t tv_chain_workspace_size(int64_t num_chains, int64_t max_len)
{
    if (num_chains < 0 || max_len < 0) return 0;
    const long long warps = (num_chains + WARP - 1) / WARP;
    return carve_chain_ws(nullptr, warps, max_len + 1, 2 * num_chains * max_len + 2 * num_chains).bytes;
}

tv_status tv_chain_solve_general(const float *d_a, const float *d_b, const float *d_wlo,
                                 const float *d_whi, const int64_t *d_offsets, int64_t num_chains,
                                 int64_t max_len, float *d_x, void *d_workspace,
                                 size_t workspace_bytes, tv_stream_t stream)
{
    clear_error();
    if (num_chains < 0 || max_len < 0 || max_len > (1LL << 24)) {
        set_error("tv_chain_solve_general: num_chains and max_len must be >= 0 (max_len <= 2^24)");
        return TV_ERR_INVALID;
    }
    if (num_chains == 0) return TV_OK;
    if (!d_b || !d_wlo || !d_whi || !d_x || !d_workspace) {
        set_error("tv_chain_solve_general: b, wlo, whi, x and workspace must not be NULL");
        return TV_ERR_INVALID;
    }
    const void *ins[4] = {d_a, d_b, d_wlo, d_whi};
    if (!d_offsets) {
        const size_t bytes = (size_t)num_chains * (size_t)max_len * sizeof(float);
        for (const void *q : ins)
            if (overlaps(d_x, bytes, q, bytes)) {
                set_error("tv_chain_solve_general: x must not overlap the inputs");
                return TV_ERR_INVALID;
            }
    } else {
        for (const void *q : ins)
            if (q == d_x) {
                set_error("tv_chain_solve_general: x must not alias the inputs");
                return TV_ERR_INVALID;
            }
    }
    const long long warps = (num_chains + WARP - 1) / WARP;
    const long long total = (long long)num_chains * max_len;
    ChainWs ws = carve_chain_ws(d_workspace, warps, max_len, 2 * total + 2 * num_chains);
    if (workspace_bytes < ws.bytes) {
        set_error("tv_chain_solve_general: workspace of %zu bytes, %zu needed", workspace_bytes,
                  ws.bytes);
        return TV_ERR_NOMEM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    tv_status st = check_cuda(cudaMemsetAsync(ws.hdr, 0, sizeof(WsHeader), s), "memset header");
    if (st != TV_OK) return st;
    GenRowsP p{d_a, d_b, d_wlo, d_whi, d_offsets, num_chains, (int)max_len, d_x, 0};
    return launch_coop(p, num_chains, (int)max_len, ws.rec, nullptr, ws.spill, ws.hdr, s, PK_CHAIN);
}

tv_status tv_chain_solve(const float *d_y, const float *d_w, float lambda,
                         const int64_t *d_offsets, int64_t num_chains, int64_t max_len,
                         float *d_x, void *d_workspace, size_t workspace_bytes,
                         tv_stream_t stream)
{
    clear_error();
    if (num_chains < 0 || max_len < 0 || max_len > (1LL << 24)) {
        set_error("tv_chain_solve: num_chains and max_len must be >= 0 (max_len <= 2^24)");
        return TV_ERR_INVALID;
    }
    if (num_chains == 0) return TV_OK;
    if (!d_y || !d_x || !d_workspace) {
        set_error("tv_chain_solve: y, x and workspace must not be NULL");
        return TV_ERR_INVALID;
    }
    if (!d_w && !(lambda >= 0.f && lambda < INFINITY)) {
        set_error("tv_chain_solve: lambda must be finite and >= 0");
        return TV_ERR_INVALID;
    }
    // Without offsets the node count is known on the host: check overlap of x with the inputs.
    if (!d_offsets) {
        const size_t bytes = (size_t)num_chains * (size_t)max_len * sizeof(float);
        if (overlaps(d_x, bytes, d_y, bytes) || overlaps(d_x, bytes, d_w, bytes)) {
            set_error("tv_chain_solve: x must not overlap y or w");
            return TV_ERR_INVALID;
        }
    } else if (d_x == d_y || (d_w && d_x == d_w)) {
        set_error("tv_chain_solve: x must not alias y or w");
        return TV_ERR_INVALID;
    }
    const long long warps = (num_chains + WARP - 1) / WARP;
    // The total node count may live on the device only; num_chains * max_len bounds it.
    const long long total = (long long)num_chains * max_len;
    // max_len + 1 record rows per warp: the middle-rooted kernel's 16 chains per warp take
    // two lanes of ceil(max_len / 2) rows each
    ChainWs ws = carve_chain_ws(d_workspace, warps, max_len + 1, 2 * total + 2 * num_chains);
    if (workspace_bytes < ws.bytes) {
        set_error("tv_chain_solve: workspace of %zu bytes, %zu needed", workspace_bytes, ws.bytes);
        return TV_ERR_NOMEM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    tv_status st = check_cuda(cudaMemsetAsync(ws.hdr, 0, sizeof(WsHeader), s), "memset header");
    if (st != TV_OK) return st;
    const bool vec_w = vec_ok(d_offsets, max_len, d_y, d_w, d_x);
    // by default, batches the fixed-shape thread kernel stages 16 bytes at a time leave
    // the warp-per-chain kernel at a smaller batch size
    const bool vec_flat = vec_w && max_len >= kHalvesMinLen && thread_split() == 2;
    const long long coop_max = coop_max_auto() && vec_flat ? kCoopMaxChainsVec : coop_max_chains();
    if (num_chains <= coop_max) {
        if (d_w) {
            CoopRowsP<true> p{d_y, d_w, 0.f, d_offsets, num_chains, (int)max_len, d_x, 0,
                              &ws.hdr->status};
            return launch_coop(p, num_chains, (int)max_len, ws.rec, nullptr, ws.spill, ws.hdr, s, PK_CHAIN);
        }
        CoopRowsP<false> p{d_y, nullptr, lambda, d_offsets, num_chains, (int)max_len, d_x, 0,
                           &ws.hdr->status};
        return launch_coop(p, num_chains, (int)max_len, ws.rec, nullptr, ws.spill, ws.hdr, s, PK_CHAIN);
    }
    // chains of 64 nodes or more: two threads per chain (twice the warps, half the steps
    // each, and a 16-entry ring that keeps every warp of a full batch resident)
    // mode 2 (default): the fixed-shape update, except per-edge weights on chains shorter
    // than kFlatMinLenW nodes that are not staged 16 bytes at a time, where the halves with
    // the scans in step (mode 1) measured faster (the flat kernel then stages every weight
    // with its own 4-byte copy)
    int split = max_len >= kHalvesMinLen ? thread_split() : 0;
    if (split == 2 && d_w && max_len < kFlatMinLenW && !vec_w) split = 1;
    if (d_w) {
        ChainRowsP<true> p{d_y, d_w, 0.f, d_offsets, num_chains, (int)max_len, d_x,
                           vec_w, 0, &ws.hdr->status};
        if (split == 2) return launch_flat(p, num_chains, (int)max_len, ws.rec, ws.spill, ws.hdr, s);
        if (split == 1) return launch_halves(p, num_chains, (int)max_len, ws.rec, ws.spill, ws.hdr, s);
        return launch_batch(p, num_chains, ws.rec, nullptr, ws.spill, ws.hdr, s);
    }
    ChainRowsP<false> p{d_y, nullptr, lambda, d_offsets, num_chains, (int)max_len, d_x,
                        vec_ok(d_offsets, max_len, d_y, nullptr, d_x), 0, &ws.hdr->status};
    if (split == 2) return launch_flat(p, num_chains, (int)max_len, ws.rec, ws.spill, ws.hdr, s);
    if (split == 1) return launch_halves(p, num_chains, (int)max_len, ws.rec, ws.spill, ws.hdr, s);
    return launch_batch(p, num_chains, ws.rec, nullptr, ws.spill, ws.hdr, s);
}

size_t tv_columns_workspace_size(int64_t H, int64_t W)
{
    if (H < 0 || W < 0) return 0;
    const long long warps = (W + WARP - 1) / WARP;
    return carve_chain_ws(nullptr, warps, H, W * (2 * H + 2)).bytes;
}

tv_status tv_chain_solve_columns(const float *d_y, const float *d_w, float lambda, int64_t H,
                                 int64_t W, int64_t ld, float *d_x, void *d_workspace,
                                 size_t workspace_bytes, tv_stream_t stream)
{
    clear_error();
    if (H < 0 || W < 0 || ld < W || H > (1LL << 24)) {
        set_error("tv_chain_solve_columns: need H, W >= 0 and ld >= W");
        return TV_ERR_INVALID;
    }
    if (H == 0 || W == 0) return TV_OK;
    if (!d_y || !d_x || !d_workspace) {
        set_error("tv_chain_solve_columns: y, x and workspace must not be NULL");
        return TV_ERR_INVALID;
    }
    if (!d_w && !(lambda >= 0.f && lambda < INFINITY)) {
        set_error("tv_chain_solve_columns: lambda must be finite and >= 0");
        return TV_ERR_INVALID;
    }
    const size_t bytes = (size_t)((H - 1) * ld + W) * sizeof(float);
    if (overlaps(d_x, bytes, d_y, bytes) || overlaps(d_x, bytes, d_w, bytes)) {
        set_error("tv_chain_solve_columns: x must not overlap y or w");
        return TV_ERR_INVALID;
    }
    const long long warps = (W + WARP - 1) / WARP;
    ChainWs ws = carve_chain_ws(d_workspace, warps, H, W * (2 * H + 2));
    if (workspace_bytes < ws.bytes) {
        set_error("tv_chain_solve_columns: workspace of %zu bytes, %zu needed", workspace_bytes,
                  ws.bytes);
        return TV_ERR_NOMEM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    tv_status st = check_cuda(cudaMemsetAsync(ws.hdr, 0, sizeof(WsHeader), s), "memset header");
    if (st != TV_OK) return st;
    if (W <= coop_max_chains()) {
        if (d_w) {
            CoopColsP<true> p{d_y, d_w, 0.f, H, W, ld, d_x};
            return launch_coop(p, W, (int)H, ws.rec, nullptr, ws.spill, ws.hdr, s, PK_CHAIN);
        }
        CoopColsP<false> p{d_y, nullptr, lambda, H, W, ld, d_x};
        return launch_coop(p, W, (int)H, ws.rec, nullptr, ws.spill, ws.hdr, s, PK_CHAIN);
    }
    if (d_w) {
        ChainColsP<true> p{d_y, d_w, 0.f, H, W, ld, d_x, vec_ok(nullptr, ld, d_y, d_w, d_x)};
        return launch_batch(p, W, ws.rec, nullptr, ws.spill, ws.hdr, s);
    }
    ChainColsP<false> p{d_y, nullptr, lambda, H, W, ld, d_x, vec_ok(nullptr, ld, d_y, nullptr, d_x)};
    return launch_batch(p, W, ws.rec, nullptr, ws.spill, ws.hdr, s);
}

tv_status tv_workspace_status(void *d_workspace, tv_stream_t stream, int *status_out,
                              int64_t *overflowed)
{
    clear_error();
    if (!d_workspace || !status_out) {
        set_error("tv_workspace_status: workspace and status_out must not be NULL");
        return TV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    WsHeader h;
    tv_status st = check_cuda(cudaMemcpyAsync(&h, d_workspace, sizeof(h), cudaMemcpyDeviceToHost, s),
                              "read header");
    if (st == TV_OK) st = check_cuda(cudaStreamSynchronize(s), "synchronize");
    if (st != TV_OK) return st;
    *status_out = (h.status & ERR_BAD_CHAIN)  ? TV_ERR_INVALID
                  : (h.status & ERR_CAPACITY) ? TV_ERR_CAPACITY
                                              : TV_OK;
    if (overflowed) *overflowed = (int64_t)h.overflowed;
    return check_cuda(cudaMemsetAsync(d_workspace, 0, sizeof(WsHeader), s), "clear header");
}

}  // extern "C"

// ------------------------------------------------------------------------------
// Chain solve for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc at all: code running inside a framework
// that has reserved the GPU's memory for its own caching allocator (a cudaMalloc
// there fails or fragments the framework's pool), and latency-critical loops that
// cannot take the implicit device synchronisation an allocation may cause. They
// pass only inputs and outputs; the scratch (the per-node records of the forward
// pass and the reserve for long message sequences) comes from this fixed array.
//
// The array lives in every GPU that loads the library, until the process exits.
// Its device address belongs to the CUDA context that is current when it is looked
// up: the address is looked up on the first call made on a device (make that first
// call before any stream capture) and again whenever that device's current context
// has changed since (after cudaDeviceReset, say), keyed by the context's unique id.
// Every call shares the array: calls that overlap on the GPU (different streams,
// or different host threads, on the same device) race on it and must be ordered
// by the caller. The header words are cleared on every call.
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr int kNoAllocMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
struct NoAllocSlot {
    void *ptr;
    unsigned long long ctx;  // id of the context the address was looked up in
};
NoAllocSlot g_noalloc[kNoAllocMaxDevices];

// Unique id of the current context (cuCtxGetId through the runtime's driver entry
// point, so that the library needs no link to the driver library); false if there is
// no current context or the driver has no such call.
bool current_context_id(unsigned long long *id)
{
    typedef int (*CtxGetId)(void *, unsigned long long *);
    static CtxGetId fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            (void)cudaGetLastError();
            return (CtxGetId) nullptr;
        }
        return (CtxGetId)f;
    }();
    return fn != nullptr && fn(nullptr, id) == 0;
}

tv_status noalloc_scratch(void **out)
{
    int dev = 0;
    tv_status st = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (st != TV_OK) return st;
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("tv_chain_solve_noalloc: device ordinal %d is not supported", dev);
        return TV_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    unsigned long long ctx = 0;
    if (g_noalloc[dev].ptr && current_context_id(&ctx) && ctx == g_noalloc[dev].ctx) {
        *out = g_noalloc[dev].ptr;
        return TV_OK;
    }
    void *p = nullptr;
    st = check_cuda(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
    if (st != TV_OK) return st;
    // without a context id the address is looked up again on every call
    g_noalloc[dev].ptr = current_context_id(&ctx) ? p : nullptr;
    g_noalloc[dev].ctx = ctx;
    *out = p;
    return TV_OK;
}

}  // namespace

extern "C" tv_status tv_chain_solve_noalloc(const float *d_y, const float *d_w, float lambda,
                                            const int64_t *d_offsets, int64_t num_chains,
                                            int64_t max_len, float *d_x, tv_stream_t stream)
{
    clear_error();
    if (num_chains < 0 || max_len < 0 || max_len > (1LL << 24)) {
        set_error("tv_chain_solve_noalloc: num_chains and max_len must be >= 0 (max_len <= 2^24)");
        return TV_ERR_INVALID;
    }
    if (num_chains == 0) return TV_OK;
    if (!d_y || !d_x) {
        set_error("tv_chain_solve_noalloc: y and x must not be NULL");
        return TV_ERR_INVALID;
    }
    if (!d_w && !(lambda >= 0.f && lambda < INFINITY)) {
        set_error("tv_chain_solve_noalloc: lambda must be finite and >= 0");
        return TV_ERR_INVALID;
    }
    if (!d_offsets) {
        const size_t bytes = (size_t)num_chains * (size_t)max_len * sizeof(float);
        if (overlaps(d_x, bytes, d_y, bytes) || overlaps(d_x, bytes, d_w, bytes)) {
            set_error("tv_chain_solve_noalloc: x must not overlap y or w");
            return TV_ERR_INVALID;
        }
    } else if (d_x == d_y || (d_w && d_x == d_w)) {
        set_error("tv_chain_solve_noalloc: x must not alias y or w");
        return TV_ERR_INVALID;
    }
    const long long warps = (num_chains + WARP - 1) / WARP;
    const long long total = (long long)num_chains * max_len;
    const size_t need = carve_chain_ws(nullptr, warps, max_len, 2 * total + 2 * num_chains).bytes;
    if (need > kNoAllocScratchBytes) {
        set_error("tv_chain_solve_noalloc: %lld chains x %lld nodes need %zu bytes of scratch, "
                  "more than the fixed %zu; use tv_chain_solve with a workspace",
                  (long long)num_chains, (long long)max_len, need, kNoAllocScratchBytes);
        return TV_ERR_INVALID;
    }
    void *scratch = nullptr;
    tv_status st = noalloc_scratch(&scratch);
    if (st != TV_OK) return st;
    ChainWs ws = carve_chain_ws(scratch, warps, max_len, 2 * total + 2 * num_chains);
    cudaStream_t s = (cudaStream_t)stream;
    st = check_cuda(cudaMemsetAsync(ws.hdr, 0, sizeof(WsHeader), s), "clear scratch header");
    if (st != TV_OK) return st;
    if (d_w) {
        ChainRowsP<true> p{d_y, d_w, 0.f, d_offsets, num_chains, (int)max_len, d_x,
                           vec_ok(d_offsets, max_len, d_y, d_w, d_x), 0, &ws.hdr->status};
        return launch_batch(p, num_chains, ws.rec, nullptr, ws.spill, ws.hdr, s);
    }
    ChainRowsP<false> p{d_y, nullptr, lambda, d_offsets, num_chains, (int)max_len, d_x,
                        vec_ok(d_offsets, max_len, d_y, nullptr, d_x), 0, &ws.hdr->status};
    return launch_batch(p, num_chains, ws.rec, nullptr, ws.spill, ws.hdr, s);
}
