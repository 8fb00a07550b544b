// Vector-Jacobian product of the chain TV prox (the backward of a
// differentiable TV layer built on eq. 1D-ROF).
//
// Away from degenerate inputs the optimality conditions of eq. 1D-ROF fix the
// solution on every maximal run S = [l..r] of equal values ("segment") as
//     x_S = mean(y_S) + (u_r - u_{l-1}) / |S|,   u_e = w_e * sign(x_{e+1} - x_e)
// at the jump edges bounding S (u = 0 past the chain ends). Hence, for an
// upstream gradient g = dL/dx,
//     dL/dy_j = mean_{i in S(j)} g_i,
//     dL/dw_e = sign_e * (mean_{S left of e} g - mean_{S right of e} g) at a jump
//               edge e, and 0 on the edges inside a segment.
// Segments are read off the forward output: the backward clip of Algorithm 2
// copies x_{i+1} into x_i whenever the clip is inactive, so fused neighbours are
// bitwise equal.
//
// One warp per chain, 32 nodes per step: a forward segmented scan of (sum, count)
// with a carry across steps yields each segment's mean at its last node; a reverse
// segmented scan spreads it over the segment. The chain's g and the means stay in
// shared memory when the chain fits, so each node is read and written once. The loads
// of kGradUnroll steps are issued together before their scans run one after another:
// with one step's loads in flight per warp, the kernel was bound by memory latency.
#include <cuda_runtime.h>

#include "tv_launch.cuh"

using namespace tvk;
using namespace tvh;

namespace {

constexpr int kGradWarps = 4;
constexpr int kGradSmemNodes = 4096;  // g and segment means of one chain: 8 bytes per node
constexpr int kGradUnroll = 4;        // steps whose loads are in flight together

struct GradArgs {
    const float *x, *g;
    const int64_t *offsets;
    long long nchains;
    int maxlen;
    float *gy, *gw;
    int smem_nodes;
};

__global__ void __launch_bounds__(kGradWarps * WARP) chain_vjp_kernel(GradArgs a, WsHeader *hdr)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & (WARP - 1);
    const int warp = threadIdx.x / WARP;
    const long long k = (long long)blockIdx.x * kGradWarps + warp;
    if (k >= a.nchains) return;
    long long start;
    int n;
    if (a.offsets) {
        const long long o0 = a.offsets[0], lo = a.offsets[k], hi = a.offsets[k + 1];
        if (lo < o0 || hi < lo || hi - lo > a.maxlen || hi - o0 > (k + 1) * (long long)a.maxlen) {
            if (lane == 0) atomicOr(&hdr->status, ERR_BAD_CHAIN);
            return;
        }
        start = lo;
        n = (int)(hi - lo);
    } else {
        start = k * (long long)a.maxlen;
        n = a.maxlen;
    }
    if (n == 0) return;
    const float *x = a.x + start, *g = a.g + start;
    float *gy = a.gy + start;
    // per-node segment means: shared memory when the chain fits, else grad_y itself
    float *mean = (n <= a.smem_nodes)
                      ? reinterpret_cast<float *>(smem_raw) + (size_t)warp * a.smem_nodes
                      : gy;
    const int nblk = (n + WARP - 1) / WARP;

    // ---- forward: segmented (sum, count); the mean lands on each segment's last node
    constexpr int U = kGradUnroll;
    float carry_s = 0.f;
    int carry_c = 0;  // open segment entering this block
    for (int b0 = 0; b0 < nblk; b0 += U) {
        float xv[U], xp[U], xn[U], gv[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int i = (b0 + q) * WARP + lane;
            const bool in = i < n;
            xv[q] = in ? x[i] : 0.f;
            xp[q] = (in && i > 0) ? x[i - 1] : 0.f;
            xn[q] = (i + 1 < n) ? x[i + 1] : 0.f;
            gv[q] = in ? g[i] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int b = b0 + q;
            if (b >= nblk) break;  // the same for every lane
            const int i = b * WARP + lane;
            const bool in = i < n;
            const float xi = xv[q];
            const float xprev = xp[q];
            const float xnext = xn[q];
            const bool head = in && (i == 0 || xi != xprev);
            const bool tail = in && (i == n - 1 || xi != xnext);
            float s = gv[q];
            // the segment of node i starts at lane hs of this step (-1: before it); the
            // sum over [max(hs, 0), lane] by the doubling scan, taking a partial sum only
            // from a lane inside the segment; the count from the lane index
            const unsigned hm = __ballot_sync(FULL, head) & (0xffffffffu >> (WARP - 1 - lane));
            const int hs = hm ? WARP - 1 - __clz(hm) : -1;
#pragma unroll
            for (int o = 1; o < WARP; o <<= 1) {
                const float s2 = __shfl_up_sync(FULL, s, o);
                if (lane - o >= (hs < 0 ? 0 : hs)) s += s2;
            }
            int c = hs < 0 ? lane + 1 + carry_c : lane - hs + 1;
            if (hs < 0) s += carry_s;
            if (tail) mean[i] = s / (float)c;
            carry_s = __shfl_sync(FULL, s, WARP - 1);
            carry_c = __shfl_sync(FULL, c, WARP - 1);
            // a segment that ended on the block's last node does not carry on
            const bool last_tail = __shfl_sync(FULL, (int)tail, WARP - 1);
            if (last_tail) {
                carry_s = 0.f;
                carry_c = 0;
            }
        }
    }
    __syncwarp();
    // ---- backward: every node takes the mean stored at its segment's last node
    // (a batch's tail means are read before any of its outputs is written: for a chain
    // longer than the shared-memory records the means live in grad_y itself, each at its
    // segment's last node, inside the step that owns that node)
    float carry_m = 0.f;
    for (int b0 = nblk - 1; b0 >= 0; b0 -= U) {
        float xv[U], xn[U], mv[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int i = (b0 - q) * WARP + lane;
            const bool in = b0 - q >= 0 && i < n;
            xv[q] = in ? x[i] : 0.f;
            xn[q] = (in && i + 1 < n) ? x[i + 1] : 0.f;
            mv[q] = (in && (i == n - 1 || xv[q] != xn[q])) ? mean[i] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int b = b0 - q;
            if (b < 0) break;  // the same for every lane
            const int i = b * WARP + lane;
            const bool in = i < n;
            const float xi = xv[q];
            const float xnext = xn[q];
            const bool tail = in && (i == n - 1 || xi != xnext);
            // the mean sits at the segment's last node: lane te of this step, or (no tail
            // at or after this lane) a later step, whose mean is the carry
            const unsigned tm = __ballot_sync(FULL, tail) & (0xffffffffu << lane);
            const int te = tm ? __ffs(tm) - 1 : lane;
            float m = __shfl_sync(FULL, mv[q], te);
            if (!tm) m = carry_m;
            const float mn = __shfl_down_sync(FULL, m, 1);
            const float mright = (lane == WARP - 1) ? carry_m : mn;  // mean of node i+1
            __syncwarp();
            if (in) {
                gy[i] = m;
                // jump edge i -> i+1: sign * (mean left - mean right); fused edges: 0
                if (a.gw && i + 1 < n)
                    a.gw[start + i] = tail ? ((xnext > xi ? 1.f : -1.f) * (m - mright)) : 0.f;
            }
            carry_m = __shfl_sync(FULL, m, 0);
        }
    }
}

}  // namespace

extern "C" tv_status tv_chain_solve_backward(const float *d_x, const float *d_grad_x,
                                             const int64_t *d_offsets, int64_t num_chains,
                                             int64_t max_len, float *d_grad_y, float *d_grad_w,
                                             void *d_workspace, size_t workspace_bytes,
                                             tv_stream_t stream)
{
    clear_error();
    if (num_chains < 0 || max_len < 0 || max_len > (1LL << 24)) {
        set_error("tv_chain_solve_backward: num_chains and max_len must be >= 0");
        return TV_ERR_INVALID;
    }
    if (num_chains == 0) return TV_OK;
    if (!d_x || !d_grad_x || !d_grad_y || !d_workspace) {
        set_error("tv_chain_solve_backward: x, grad_x, grad_y and workspace must not be NULL");
        return TV_ERR_INVALID;
    }
    if (d_grad_y == d_x || d_grad_y == d_grad_x || (d_grad_w && (d_grad_w == d_x ||
                                                                 d_grad_w == d_grad_x ||
                                                                 d_grad_w == d_grad_y))) {
        set_error("tv_chain_solve_backward: outputs must not alias the inputs or each other");
        return TV_ERR_INVALID;
    }
    if (workspace_bytes < sizeof(WsHeader)) {
        set_error("tv_chain_solve_backward: workspace of %zu bytes, %zu needed", workspace_bytes,
                  sizeof(WsHeader));
        return TV_ERR_NOMEM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    WsHeader *hdr = static_cast<WsHeader *>(d_workspace);
    tv_status st = check_cuda(cudaMemsetAsync(hdr, 0, sizeof(WsHeader), s), "memset header");
    if (st != TV_OK) return st;
    const int smem_nodes = max_len <= kGradSmemNodes ? (int)max_len : 0;
    const size_t smem = (size_t)kGradWarps * smem_nodes * sizeof(float);
    st = check_cuda(cudaFuncSetAttribute(chain_vjp_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    "cudaFuncSetAttribute");
    if (st != TV_OK) return st;
    GradArgs a{d_x, d_grad_x, d_offsets, num_chains, (int)max_len, d_grad_y, d_grad_w, smem_nodes};
    const long long blocks = (num_chains + kGradWarps - 1) / kGradWarps;
    const bool prof = prof_on();
    if (prof) prof_mark(PK_GRAD, s, true);
    chain_vjp_kernel<<<(unsigned)blocks, kGradWarps * WARP, smem, s>>>(a, hdr);
    st = check_cuda(cudaGetLastError(), "backward kernel launch");
    if (st == TV_OK) note_launch();
    if (prof) prof_mark(PK_GRAD, s, false);
    return st;
}
