// Kernels of the dual warm-start network: a small 3x3 convolutional net that
// maps a noisy image and its weight lambda to an initial dual of the 2D primal-
// dual iteration (the warm start y^0 of eq. pd). The network is not part of the
// paper; the 2D solver accepts any y^0 and still converges.
//
// Tensors are NHWC with channel counts of 16 or 32 (zero-padded). Convolutions
// are implicit GEMMs on BF16 tensor cores (mma.sync m16n8k16, FP32 accumulate):
//   forward:        M = pixels, N = Cout, K = 9 * Cin
//   backward data:  the same with the kernel flipped and Cin/Cout swapped
//   backward weight: M = Cout, N = 9 * Cin, K = pixels (persistent blocks, FP32
//                    partial tiles, atomics into the FP32 gradient)
// Each block of the two pixel-major kernels computes an 8 x 16 pixel tile for all
// output channels from a zero-padded 10 x 18 input patch in shared memory; A and B
// fragments are read with ldmatrix from rows padded by 16 bytes (conflict-free).
#include <atomic>
#include <cstdint>
#include <cstring>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "tv_launch.cuh"

using namespace tvk;
using namespace tvh;

namespace {

constexpr int TH = 8, TW = 16;  // output tile (rows x cols) of one block
constexpr int PH = TH + 2, PW = TW + 2;
constexpr int NTHR = 128;       // 4 warps, 2 tile rows each

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2,
                                        unsigned &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(unsigned addr, unsigned &r0, unsigned &r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r0), "=r"(r1)
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2,
                                          unsigned &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_t(unsigned addr, unsigned &r0, unsigned &r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r0), "=r"(r1)
                 : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Load the zero-padded (TH+2) x (TW+2) x C input patch of tile (ty, tx) of image b.
template <int C>
__device__ __forceinline__ void load_patch(__nv_bfloat16 *patch, const __nv_bfloat16 *X, int b,
                                           int H, int W, int y0, int x0)
{
    constexpr int PS = C + 8;   // padded pixel stride (bf16)
    constexpr int V = C / 8;    // 16-byte vectors per pixel
    for (int t = threadIdx.x; t < PH * PW * V; t += blockDim.x) {
        const int v = t % V, pix = t / V;
        const int py = pix / PW, px = pix % PW;
        const int gy = y0 + py - 1, gx = x0 + px - 1;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (gy >= 0 && gy < H && gx >= 0 && gx < W)
            val = *reinterpret_cast<const uint4 *>(X + (((long long)b * H + gy) * W + gx) * C + v * 8);
        *reinterpret_cast<uint4 *>(patch + pix * PS + v * 8) = val;
    }
}

// The same patch with 16-byte asynchronous copies (zero-filled outside the image).
__device__ __forceinline__ void cp_async16_zfill(void *smem, const void *gmem, bool valid)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit_net() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_net()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int C>
__device__ __forceinline__ void load_patch_async(__nv_bfloat16 *patch, const __nv_bfloat16 *X,
                                                 int b, int H, int W, int y0, int x0)
{
    constexpr int PS = C + 8;
    constexpr int V = C / 8;
    for (int t = threadIdx.x; t < PH * PW * V; t += blockDim.x) {
        const int v = t % V, pix = t / V;
        const int py = pix / PW, px = pix % PW;
        const int gy = y0 + py - 1, gx = x0 + px - 1;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        const __nv_bfloat16 *src = in ? X + (((long long)b * H + gy) * W + gx) * C + v * 8 : X;
        cp_async16_zfill(patch + pix * PS + v * 8, src, in);
    }
}

// Output-tile convolution, persistent: each block loads the weights once and walks the
// 8 x 16 output tiles blockIdx.x, +gridDim.x, ..., prefetching the next tile's input
// patch with asynchronous copies (double buffer) while the tensor cores work on the
// current one. MODE 0: forward, out = conv + bias, optional ReLU; writes the FP32
// pre-activation (if pre_out) and the BF16 activation (if act_out). MODE 1: backward
// data: out = conv (weights already flipped/transposed), times the ReLU mask
// (mask_pre > 0) of the layer below; writes BF16.
template <int CIN, int COUT>
constexpr size_t conv_persist_smem()
{
    return sizeof(__nv_bfloat16) * ((size_t)COUT * (9 * CIN + 8) + 2 * (size_t)PH * PW * (CIN + 8));
}

template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(NTHR)
    conv3x3_persist(const __nv_bfloat16 *X, int B, int H, int W, const __nv_bfloat16 *Wt,
                    const float *bias, int relu, const float *mask_pre, float *pre_out,
                    __nv_bfloat16 *act_out)
{
    constexpr int PS = CIN + 8;
    constexpr int K = 9 * CIN;
    constexpr int KS = K + 8;
    constexpr int NT = COUT / 8;
    constexpr int PATCH = PH * PW * PS;
    extern __shared__ __align__(16) unsigned char smem_net[];
    __nv_bfloat16 *wsm = reinterpret_cast<__nv_bfloat16 *>(smem_net);
    __nv_bfloat16 *pbuf = wsm + COUT * KS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
    const int per_img = tiles_x * tiles_y;
    const long long ntiles = (long long)B * per_img;
    auto origin = [&](long long tile, int &b, int &y0, int &x0) {
        b = (int)(tile / per_img);
        const int rem = (int)(tile - (long long)b * per_img);
        y0 = (rem / tiles_x) * TH;
        x0 = (rem % tiles_x) * TW;
    };
    long long tile = blockIdx.x;
    if (tile < ntiles) {
        int b, y0, x0;
        origin(tile, b, y0, x0);
        load_patch_async<CIN>(pbuf, X, b, H, W, y0, x0);
    }
    cp_async_commit_net();
    for (int t = threadIdx.x; t < COUT * (K / 8); t += blockDim.x) {
        const int n = t / (K / 8), v = t % (K / 8);
        *reinterpret_cast<uint4 *>(wsm + n * KS + v * 8) =
            *reinterpret_cast<const uint4 *>(Wt + (long long)n * K + v * 8);
    }
    const int arow = lane & 15;
    const int acol = (lane >> 4) * 8;
    const int brow = lane & 7;
    const int bcol = ((lane >> 3) & 1) * 8;
    const int g = lane >> 2, tq = lane & 3;
    int buf = 0;
    for (; tile < ntiles; tile += gridDim.x) {
        const long long next = tile + gridDim.x;
        if (next < ntiles) {
            int b, y0, x0;
            origin(next, b, y0, x0);
            load_patch_async<CIN>(pbuf + (buf ^ 1) * PATCH, X, b, H, W, y0, x0);
        }
        cp_async_commit_net();
        cp_async_wait_net<1>();
        __syncthreads();
        const __nv_bfloat16 *patch = pbuf + buf * PATCH;
        float acc[2][NT][4];
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int j = 0; j < NT; ++j) acc[m][j][0] = acc[m][j][1] = acc[m][j][2] = acc[m][j][3] = 0.f;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap % 3;
#pragma unroll
            for (int c0 = 0; c0 < CIN; c0 += 16) {
                const int k0 = tap * CIN + c0;
                unsigned bf[NT][2];
#pragma unroll
                for (int j = 0; j < NT; ++j)
                    ldsm_x2(smem_u32(wsm + (j * 8 + brow) * KS + k0 + bcol), bf[j][0], bf[j][1]);
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const int py = warp * 2 + m + ky, px = arow + kx;
                    unsigned a0, a1, a2, a3;
                    ldsm_x4(smem_u32(patch + (py * PW + px) * PS + c0 + acol), a0, a1, a2, a3);
#pragma unroll
                    for (int j = 0; j < NT; ++j) mma_bf16(acc[m][j], a0, a1, a2, a3, bf[j][0], bf[j][1]);
                }
            }
        }
        int b, y0, x0;
        origin(tile, b, y0, x0);
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int y = y0 + warp * 2 + m;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int x = x0 + g + half * 8;
                if (y >= H || x >= W) continue;
                const long long base = (((long long)b * H + y) * W + x) * COUT;
#pragma unroll
                for (int j = 0; j < NT; ++j) {
                    const int co = j * 8 + tq * 2;
                    float v0 = acc[m][j][half * 2 + 0], v1 = acc[m][j][half * 2 + 1];
                    if (MODE == 0) {
                        if (bias) {
                            v0 += bias[co];
                            v1 += bias[co + 1];
                        }
                        if (pre_out) *reinterpret_cast<float2 *>(pre_out + base + co) = make_float2(v0, v1);
                        if (relu) {
                            v0 = fmaxf(v0, 0.f);
                            v1 = fmaxf(v1, 0.f);
                        }
                    } else {
                        const float2 mp = *reinterpret_cast<const float2 *>(mask_pre + base + co);
                        v0 = mp.x > 0.f ? v0 : 0.f;
                        v1 = mp.y > 0.f ? v1 : 0.f;
                    }
                    if (act_out)
                        *reinterpret_cast<__nv_bfloat162 *>(act_out + base + co) = __floats2bfloat162_rn(v0, v1);
                }
            }
        }
        __syncthreads();  // every warp is done with this buffer before it is refilled
        buf ^= 1;
    }
    cp_async_wait_net<0>();
}

// Partial sums of dW[co][tap][ci] = sum over pixels p of dY[p][co] * X[p + tap][ci]
// and db[co] = sum_p dY[p][co]. Each block walks tiles blockIdx.x, +gridDim.x, ...,
// keeps its partial dW in registers (warp w owns the n8 column tiles w, w+4, ... of
// N = 9 * CIN; both m16 tiles (co 0..31) or one (co 0..15)) and stores it, with its
// partial db, to row blockIdx.x of P (row length 9 * CIN * COUT + COUT); the rows
// are summed in a fixed order by wgrad_reduce, so the result is deterministic.
template <int CIN, int COUT>
__global__ void __launch_bounds__(NTHR)
    conv3x3_wgrad(const __nv_bfloat16 *X, const __nv_bfloat16 *dY, int B, int H, int W,
                  float *P)
{
    constexpr int PS = CIN + 8;
    constexpr int DS = COUT + 8;
    constexpr int N = 9 * CIN;
    constexpr int NT = N / 8;
    constexpr int NTW = (NT + 3) / 4;   // column tiles per warp
    constexpr int MT = COUT / 16;
    __shared__ __align__(16) __nv_bfloat16 patch[PH * PW * PS];
    __shared__ __align__(16) __nv_bfloat16 dys[TH * TW * DS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
    const long long ntiles = (long long)B * tiles_x * tiles_y;
    float acc[MT][NTW][4];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int j = 0; j < NTW; ++j) acc[m][j][0] = acc[m][j][1] = acc[m][j][2] = acc[m][j][3] = 0.f;
    float bsum = 0.f;  // thread t < COUT sums channel t
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = (int)(tile / (tiles_x * tiles_y));
        const int rem = (int)(tile % (tiles_x * tiles_y));
        const int y0 = (rem / tiles_x) * TH, x0 = (rem % tiles_x) * TW;
        __syncthreads();
        load_patch<CIN>(patch, X, b, H, W, y0, x0);
        for (int t = threadIdx.x; t < TH * TW * (COUT / 8); t += blockDim.x) {
            const int v = t % (COUT / 8), pix = t / (COUT / 8);
            const int yy = y0 + pix / TW, xx = x0 + pix % TW;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (yy < H && xx < W)
                val = *reinterpret_cast<const uint4 *>(dY + (((long long)b * H + yy) * W + xx) * COUT + v * 8);
            *reinterpret_cast<uint4 *>(dys + pix * DS + v * 8) = val;
        }
        __syncthreads();
        if (threadIdx.x < COUT)
            for (int pix = 0; pix < TH * TW; ++pix) bsum += __bfloat162float(dys[pix * DS + threadIdx.x]);
        // K loop over the 128 pixels of the tile, 16 at a time (one tile row)
#pragma unroll 1
        for (int r = 0; r < TH; ++r) {
            // A = dY^T (m = co, k = pixel): transposed 8x8 loads of dys rows r*16 .. r*16+15
            unsigned af[MT][4];
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                // matrices: (co 0-7, px 0-7), (co 8-15, px 0-7), (co 0-7, px 8-15), (co 8-15, px 8-15)
                const int mat = lane >> 3, rr = lane & 7;
                const int pix = r * TW + (mat >> 1) * 8 + rr;
                const int co = m * 16 + (mat & 1) * 8;
                ldsm_x4_t(smem_u32(dys + pix * DS + co), af[m][0], af[m][1], af[m][2], af[m][3]);
            }
#pragma unroll
            for (int j = 0; j < NTW; ++j) {
                const int nt = warp + 4 * j;
                if (nt < NT) {
                    // B (k = pixel, n = (tap, ci)) from the patch: rows = pixels, ci contiguous
                    const int n0 = nt * 8, tap = n0 / CIN, ci = n0 % CIN;
                    const int ky = tap / 3, kx = tap % 3;
                    const int mat = (lane >> 3) & 1, rr = lane & 7;
                    const int px = mat * 8 + rr;  // pixel within the 16-pixel row
                    unsigned b0, b1;
                    ldsm_x2_t(smem_u32(patch + ((r + ky) * PW + px + kx) * PS + ci), b0, b1);
#pragma unroll
                    for (int m = 0; m < MT; ++m)
                        mma_bf16(acc[m][j], af[m][0], af[m][1], af[m][2], af[m][3], b0, b1);
                }
            }
        }
    }
    // store the block's partial gradient
    float *row = P + (long long)blockIdx.x * (COUT * N + COUT);
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int j = 0; j < NTW; ++j) {
            const int nt = warp + 4 * j;
            if (nt >= NT) continue;
            const int n = nt * 8 + tq * 2;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int co = m * 16 + g + half * 8;
                *reinterpret_cast<float2 *>(row + co * N + n) =
                    make_float2(acc[m][j][half * 2], acc[m][j][half * 2 + 1]);
            }
        }
    if (threadIdx.x < COUT) row[COUT * N + threadIdx.x] = bsum;
}

// dW[e] += sum_b P[b][e] (e < nw) and db[e - nw] += sum_b P[b][e] (nw <= e < stride),
// summed in a fixed order: 32 consecutive e per block row of threads, 8 interleaved
// groups of b per column, the 8 group sums combined in order.
constexpr int RED_E = 32, RED_G = 8;
__global__ void __launch_bounds__(RED_E * RED_G)
    wgrad_reduce(const float *P, int nblocks, int stride, int nw, float *dW, float *db)
{
    __shared__ float part[RED_G][RED_E];
    const int te = threadIdx.x % RED_E, tg = threadIdx.x / RED_E;
    const int e = blockIdx.x * RED_E + te;
    float sum = 0.f;
    if (e < stride) {
#pragma unroll 4
        for (int b = tg; b < nblocks; b += RED_G) sum += P[(long long)b * stride + e];
    }
    part[tg][te] = sum;
    __syncthreads();
    if (tg == 0 && e < stride) {
        float tot = 0.f;
#pragma unroll
        for (int q = 0; q < RED_G; ++q) tot += part[q][te];
        if (e < nw) dW[e] += tot;
        else if (db) db[e - nw] += tot;
    }
}

// Blocks of the weight-gradient kernel for a B x H x W batch.
long long wgrad_blocks(int B, int H, int W)
{
    const long long ntiles = (long long)B * ((W + TW - 1) / TW) * ((H + TH - 1) / TH);
    return std::min<long long>(4LL * sm_count_current(), ntiles);
}

template <int CIN, int COUT, int MODE>
tv_status launch_conv(const __nv_bfloat16 *X, int B, int H, int W, const __nv_bfloat16 *Wt,
                      const float *bias, int relu, const float *mask_pre, float *pre_out,
                      __nv_bfloat16 *act_out, cudaStream_t s)
{
    auto kern = conv3x3_persist<CIN, COUT, MODE>;
    constexpr size_t smem = conv_persist_smem<CIN, COUT>();
    static int per_sm = 0;  // resident blocks per SM (occupancy, computed once per kernel)
    if (per_sm == 0) {
        tv_status st0 = check_cuda(
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
            "cudaFuncSetAttribute");
        if (st0 != TV_OK) return st0;
        st0 = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                              (int)cudaSharedmemCarveoutMaxShared),
                         "cudaFuncSetAttribute");
        if (st0 != TV_OK) return st0;
        int b = 0;
        st0 = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, NTHR, smem),
                         "occupancy");
        if (st0 != TV_OK) return st0;
        per_sm = b < 1 ? 1 : b;
    }
    const long long ntiles = (long long)B * ((W + TW - 1) / TW) * ((H + TH - 1) / TH);
    long long blocks = (long long)per_sm * sm_count_current();
    if (blocks > ntiles) blocks = ntiles;
    kern<<<(unsigned)blocks, NTHR, smem, s>>>(X, B, H, W, Wt, bias, relu, mask_pre, pre_out,
                                                act_out);
    tv_status st = check_cuda(cudaGetLastError(), "conv launch");
    if (st == TV_OK) note_launch();
    return st;
}

template <int CIN, int COUT>
tv_status launch_wgrad(const __nv_bfloat16 *X, const __nv_bfloat16 *dY, int B, int H, int W,
                       float *dW, float *db, float *P, cudaStream_t s)
{
    const long long blocks = wgrad_blocks(B, H, W);
    conv3x3_wgrad<CIN, COUT><<<(unsigned)blocks, NTHR, 0, s>>>(X, dY, B, H, W, P);
    tv_status st = check_cuda(cudaGetLastError(), "weight-gradient launch");
    if (st != TV_OK) return st;
    note_launch();
    constexpr int nw = COUT * 9 * CIN, stride = nw + COUT;
    wgrad_reduce<<<(stride + RED_E - 1) / RED_E, RED_E * RED_G, 0, s>>>(P, (int)blocks, stride, nw,
                                                                        dW, db);
    st = check_cuda(cudaGetLastError(), "weight-gradient reduction");
    if (st == TV_OK) note_launch();
    return st;
}

bool valid_channels(int cin, int cout)
{
    return (cin == 16 || cin == 32) && (cout == 16 || cout == 32);
}

// ---------------------------------------------------------------- elementwise --
// Head of the network: p_v = lam * tanh(o) on vertical edges (rows 0..H-2), and the
// dual y = D_v^T p_v (y[r] = p[r-1] - p[r], p[-1] = p[H-1] = 0), always feasible
// for |p_v| <= lam. With a target, also the loss sum (y - t)^2 / N (accumulated
// into *loss) and the gradient with respect to o (channel 0 of a 16-channel
// BF16 tensor, other channels zero).
__global__ void __launch_bounds__(256)
    dual_head(const float *o, int B, int H, int W, const float *lam, const float *target, float *y,
              float *loss_part, float inv_count)
{
    const long long HW = (long long)H * W;
    const long long N = (long long)B * HW;
    const long long stride = (long long)gridDim.x * blockDim.x;
    float lsum = 0.f;
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < N) {
        // image b, row r and column c of q, advanced along the grid-stride walk by the
        // same decomposition of the stride (one carry per level)
        int b = (int)(q / HW);
        const long long rem = q - (long long)b * HW;
        int r = (int)(rem / W), c = (int)(rem - (long long)r * W);
        const int sb = (int)(stride / HW);
        const long long srem = stride - (long long)sb * HW;
        const int sr = (int)(srem / W), sc = (int)(srem - (long long)sr * W);
        for (; q < N; q += stride) {
            const float L = lam[b];
            auto pv = [&](long long qq, int rr) -> float {
                return (rr >= 0 && rr < H - 1) ? L * tanhf(o[qq * 16]) : 0.f;
            };
            const float yv = pv(q - W, r - 1) - pv(q, r);
            if (y) y[q] = yv;
            if (target) {
                const float e = yv - target[q];
                lsum += e * e;
            }
            c += sc;
            r += sr;
            b += sb;
            if (c >= W) {
                c -= W;
                ++r;
            }
            if (r >= H) {
                r -= H;
                ++b;
            }
        }
    }
    if (target && loss_part) {
        __shared__ float wsum[8];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = lsum;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += wsum[q];
            loss_part[blockIdx.x] = t * inv_count;
        }
    }
}

// y = D_v^T p for p already on the vertical edges (0 on each image's last row):
// y[r] = p[r-1] - p[r], p[-1] = 0.
// Blocks along x cover a row's columns; blocks along y walk the B*H rows.
__global__ void __launch_bounds__(256) head_from_p(const float *p, long long rows, int H, int W, float *y)
{
    pdl_enter();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    int r = (int)(blockIdx.y % (unsigned)H);  // row within its image
    const int dr = (int)(gridDim.y % (unsigned)H);
    for (long long row = blockIdx.y; row < rows; row += gridDim.y) {
        const long long q = row * W + x;
        y[q] = (r > 0 ? p[q - W] : 0.f) - p[q];
        r += dr;
        if (r >= H) r -= H;
    }
}

// *loss = sum of n block partials, in a fixed order (one block).
__global__ void __launch_bounds__(256) sum_partials(const float *part, int n, float *loss)
{
    __shared__ float s[256];
    float t = 0.f;
    for (int i = threadIdx.x; i < n; i += 256) t += part[i];
    s[threadIdx.x] = t;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = s[0];
}

// d loss / d o at every pixel: dL/dp[r] = dL/dy[r+1] - dL/dy[r] for r < H-1 (0 on the
// last row), dL/dy = 2 (y - t) / count, times lam (1 - tanh(o)^2).
__global__ void dual_head_grad(const float *o, int B, int H, int W, const float *lam,
                               const float *y, const float *target, __nv_bfloat16 *d_o,
                               float inv_count)
{
    const long long N = (long long)B * H * W;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < N;
         q += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(q / ((long long)H * W));
        const int r = (int)((q % ((long long)H * W)) / W);
        float g = 0.f;
        if (r < H - 1) {
            const float dy_next = 2.f * (y[q + W] - target[q + W]) * inv_count;
            const float dy_here = 2.f * (y[q] - target[q]) * inv_count;
            const float th = tanhf(o[q * 16]);
            g = (dy_next - dy_here) * lam[b] * (1.f - th * th);
        }
        __nv_bfloat16 *dst = d_o + q * 16;
        dst[0] = __float2bfloat16(g);
#pragma unroll
        for (int c = 1; c < 16; ++c) dst[c] = __float2bfloat16(0.f);
    }
}

// Network input: channel 0 the image, channel 1 its lambda, 2..15 zero (BF16 NHWC).
// Image b of the batch is blockIdx.y. Each pixel's 16 channels (32 bytes: the image,
// lambda, 14 zeros) go out as two 16-byte stores when x is 16-byte aligned.
__global__ void pack_input(const float *f, int H, int W, const float *lam, __nv_bfloat16 *x,
                           bool vec)
{
    const long long HW = (long long)H * W;
    const int b = blockIdx.y;
    const float *fb = f + (long long)b * HW;
    __nv_bfloat16 *xb = x + (long long)b * HW * 16;
    const __nv_bfloat16 lb = __float2bfloat16(lam[b]);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < HW; q += stride) {
        const __nv_bfloat162 p01 = __halves2bfloat162(__float2bfloat16(fb[q]), lb);
        if (vec) {
            uint4 *d = reinterpret_cast<uint4 *>(xb + q * 16);
            d[0] = make_uint4(*reinterpret_cast<const unsigned *>(&p01), 0u, 0u, 0u);
            d[1] = make_uint4(0u, 0u, 0u, 0u);
        } else {
            __nv_bfloat16 *dst = xb + q * 16;
            dst[0] = p01.x;
            dst[1] = p01.y;
#pragma unroll
            for (int c = 2; c < 16; ++c) dst[c] = __float2bfloat16(0.f);
        }
    }
}

// Adam step with FP32 master weights and a BF16 copy for the forward pass.
__global__ void adam_step(float *w, float *m, float *v, float *g, long long n, float lr,
                          float b1, float b2, float eps, float bc1, float bc2, __nv_bfloat16 *w16)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        g[i] = 0.f;  // ready for the next accumulation
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        w[i] = wi;
        if (w16) w16[i] = __float2bfloat16(wi);
    }
}

// Flip a kernel and swap its channel roles: Wf[ci][tap'][co] = W[co][8 - tap'][ci]
// (the weights of the backward-data convolution).
__global__ void flip_weights(const __nv_bfloat16 *Wt, int cin, int cout, __nv_bfloat16 *Wf)
{
    const int n = cin * 9 * cout;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int co = i % cout, tap = (i / cout) % 9, ci = i / (cout * 9);
        Wf[i] = Wt[((long long)co * 9 + (8 - tap)) * cin + ci];
    }
}

int ew_blocks(long long n) { return (int)std::min<long long>((n + 255) / 256, 8LL * sm_count_current()); }

// ------------------------------------------- forward on tcgen05 (TMEM accumulators) --
// The forward convolution as tcgen05.mma instructions: one block computes 128
// consecutive output pixels of one image row (M = 128, N = COUT, K = 9 * CIN) into a
// TMEM accumulator of COUT FP32 columns. Operands are in shared memory in the
// canonical K-major layout without swizzle (8-row x 16-byte core matrices):
//   A: the three input rows y-1, y, y+1 over pixels x0-1 .. x0+128 (zero outside the
//      image), one region of 130 pixels x 16 bytes per 8-channel group; the operand of
//      tap (dy, dx) is the row-dy region started dx+1 pixels in (16 bytes per pixel),
//      so the nine taps need no copies;
//   B: the weights of every tap, [tap][8-channel group][COUT][8], loaded once per block.
// One thread issues the 9 * CIN / 16 MMAs and commits them to an mbarrier; the four
// warps then read their 32 TMEM lanes (pixels) with tcgen05.ld, add the bias, apply the
// ReLU and store. Blocks are persistent over the tiles.
constexpr int TC_M = 128;           // pixels per tile
constexpr int TC_P = TC_M + 2;      // staged pixels per row
constexpr int TC_REG = TC_P * 16;   // bytes of one (row, 8-channel group) region
constexpr unsigned kTcSpin = 1u << 26;  // mbarrier polls before a wait gives up

__device__ unsigned g_tc_timeouts;  // waits that gave up (their tiles are not written)

template <int CIN, int COUT>
constexpr size_t conv_tc_smem()
{
    return 1024 + (size_t)2 * 3 * (CIN / 8) * TC_REG + (size_t)9 * COUT * CIN * 2 + 64;  // + 2 mbarriers
}

__device__ __forceinline__ uint64_t tc_desc(unsigned saddr, unsigned lbo, unsigned sbo)
{
    // start >> 4 (bits 0-13), leading-dimension byte offset >> 4 (16-29), stride byte
    // offset >> 4 (32-45), descriptor version 1 (46-47), no swizzle (61-63 = 0)
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool tc_wait(unsigned mbar, unsigned phase)
{
    for (unsigned it = 0; it < kTcSpin; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <int N>
__device__ __forceinline__ void tc_ld(unsigned taddr, float (&v)[N])
{
    static_assert(N == 16 || N == 32, "tcgen05.ld of 16 or 32 columns");
    uint32_t r[N];
    if constexpr (N == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
            "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
              "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
              "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
              "=r"(r[31])
            : "r"(taddr));
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
            "%14,%15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = __uint_as_float(r[q]);
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(NTHR)
    conv3x3_tc(const __nv_bfloat16 *X, int B, int H, int W, const __nv_bfloat16 *Wt,
               const float *bias, int relu, float *pre_out, __nv_bfloat16 *act_out)
{
    constexpr int KG = CIN / 8;
    constexpr int ABYTES = 3 * KG * TC_REG;
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    unsigned char *abuf = smem_tc;                 // two A buffers
    unsigned char *bbuf = abuf + 2 * ABYTES;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(bbuf + 9 * COUT * CIN * 2);  // two
    unsigned *tslot = reinterpret_cast<unsigned *>(mbar + 2);
    const unsigned a_s = smem_u32(abuf), b_s = smem_u32(bbuf), mb_s = smem_u32(mbar);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = (W + TC_M - 1) / TC_M;
    const long long ntiles = (long long)B * H * tiles_x;

    // the three input rows of a tile (zero outside the image) into buffer `nb`
    auto stage = [&](long long tile, int nb) {
        const int tx = (int)(tile % tiles_x);
        const long long row = tile / tiles_x;  // b * H + y
        const int y = (int)(row % H), b = (int)(row / H);
        const int x0 = tx * TC_M;
        unsigned char *dst = abuf + nb * ABYTES;
        for (int t = tid; t < 3 * KG * TC_P; t += NTHR) {
            const int pix = t % TC_P, g = (t / TC_P) % KG, dyi = t / (TC_P * KG);
            const int gy = y + dyi - 1, gx = x0 + pix - 1;
            const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
            const __nv_bfloat16 *src = in ? X + (((long long)b * H + gy) * W + gx) * CIN + g * 8 : X;
            cp_async16_zfill(dst + (dyi * KG + g) * TC_REG + pix * 16, src, in);
        }
    };
    constexpr uint32_t idesc = tc_idesc(TC_M, COUT);
    // the 9 * CIN / 16 MMAs of a tile from A buffer `nb` into accumulator `acc_col`
    auto issue = [&](int nb, unsigned tmem_acc, unsigned mbar_addr) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const unsigned a0 = a_s + nb * ABYTES;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int dyi = tap / 3, dxi = tap % 3;
#pragma unroll
            for (int ks = 0; ks < KG / 2; ++ks) {
                const uint64_t ad = tc_desc(a0 + (dyi * KG + 2 * ks) * TC_REG + dxi * 16, TC_REG, 128);
                const uint64_t bd = tc_desc(b_s + (tap * KG + 2 * ks) * COUT * 16, COUT * 16, 128);
                const unsigned acc = (tap | ks) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_acc),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar_addr)
            : "memory");
    };

    long long tile = blockIdx.x;
    if (tile < ntiles) stage(tile, 0);
    cp_async_commit_net();
    // weights: [tap][group][co][8 channels]; bias in registers
    for (int t = tid; t < 9 * KG * COUT; t += NTHR) {
        const int co = t % COUT, g = (t / COUT) % KG, tap = t / (COUT * KG);
        *reinterpret_cast<uint4 *>(bbuf + ((tap * KG + g) * COUT + co) * 16) =
            *reinterpret_cast<const uint4 *>(Wt + ((long long)co * 9 + tap) * CIN + g * 8);
    }
    float bv[COUT];
#pragma unroll
    for (int c = 0; c < COUT; ++c) bv[c] = bias ? bias[c] : 0.f;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb_s) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb_s + 8) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        // two accumulators of 32 columns: the MMAs of a tile overlap the previous tile's epilogue
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;\n" ::"r"(
                         smem_u32(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = *tslot;

    unsigned phase[2] = {0u, 0u};
    long long prev = -1;  // the tile whose accumulator awaits its epilogue
    int i = 0;
    bool bad = false;
    auto epilogue = [&](long long t, int slot) {
        float v[COUT];
        tc_ld<COUT>(tmem + (unsigned)(slot * 32) + ((unsigned)(warp * 32) << 16), v);
        const int tx = (int)(t % tiles_x);
        const long long row = t / tiles_x;
        const int x = tx * TC_M + warp * 32 + lane;
        if (x < W) {
            const long long base = (row * W + x) * COUT;
#pragma unroll
            for (int c = 0; c < COUT; c += 4) {
                float4 q = make_float4(v[c] + bv[c], v[c + 1] + bv[c + 1], v[c + 2] + bv[c + 2],
                                       v[c + 3] + bv[c + 3]);
                if (pre_out) *reinterpret_cast<float4 *>(pre_out + base + c) = q;
                if (relu) {
                    q.x = fmaxf(q.x, 0.f);
                    q.y = fmaxf(q.y, 0.f);
                    q.z = fmaxf(q.z, 0.f);
                    q.w = fmaxf(q.w, 0.f);
                }
                if (act_out) {
                    const __nv_bfloat162 lo = __floats2bfloat162_rn(q.x, q.y);
                    const __nv_bfloat162 hi = __floats2bfloat162_rn(q.z, q.w);
                    uint2 u;
                    u.x = *reinterpret_cast<const unsigned *>(&lo);
                    u.y = *reinterpret_cast<const unsigned *>(&hi);
                    *reinterpret_cast<uint2 *>(act_out + base + c) = u;
                }
            }
        }
    };
    for (; tile < ntiles; tile += gridDim.x, ++i) {
        const int cur = i & 1;
        cp_async_wait_net<0>();  // this tile's rows
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) issue(cur, tmem + (unsigned)(cur * 32), mb_s + 8u * cur);
        if (prev >= 0) {
            // the previous tile's MMAs: done before its rows' buffer is refilled
            const bool ok = tc_wait(mb_s + 8u * (cur ^ 1), phase[cur ^ 1]);
            phase[cur ^ 1] ^= 1u;
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
        }
        const long long next = tile + gridDim.x;
        if (next < ntiles) stage(next, cur ^ 1);
        cp_async_commit_net();
        if (prev >= 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            epilogue(prev, cur ^ 1);
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        prev = tile;
    }
    if (!bad && prev >= 0) {
        const int slot = (i - 1) & 1;
        const bool ok = tc_wait(mb_s + 8u * slot, phase[slot]);
        if (__syncthreads_or(!ok)) {
            bad = true;
        } else {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            epilogue(prev, slot);
        }
    }
    if (bad && tid == 0) atomicAdd(&g_tc_timeouts, 1u);
    cp_async_wait_net<0>();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;\n" ::"r"(tmem) : "memory");
}

// ---------------------- forward on tcgen05, fed by TMA, with warp roles (tensor path 2) --
// The convolution as one GEMM per input row rather than per output row. Output row y is
// the sum over dy of input row y - 1 + dy times the weights W(dy, .); equivalently input
// row r feeds output rows r + 1, r and r - 1 through W(0, .), W(1, .) and W(2, .). So for
// each input row, shift dx and K step, one MMA with A = the row's 128 pixels from
// x0 - 1 + dx (M = 128, K = 16) and B = [W(0, dx) | W(1, dx) | W(2, dx)] (N = 3 COUT)
// adds into the TMEM accumulators of those three output rows at once, which lie side by
// side: output row o (counted along the block's rows) owns accumulator block
// TW_R - 1 - (o mod TW_R) of COUT columns, so the blocks of o + 1, o, o - 1 are
// consecutive. Where they wrap around the ring the MMA is split in two. 9 CIN / 16 MMAs
// of N = COUT per output row become 3 CIN / 16 (a little more at the wraps) of N = 3 COUT;
// a tcgen05 MMA of M = 128 and K = 16 costs nearly the same for N = 16 .. 96, so the
// count of MMAs is what sets the time. The MMAs always accumulate: the blocks start at
// zero and the epilogue zeroes each one after reading it.
// The tiles are grouped in chunks of up to L consecutive rows of one 128-pixel column of
// one image; a block takes chunks blockIdx.x, + gridDim.x, .. and walks each top-down, so
// that a chunk of n output rows reads its n + 2 input rows once each, through a ring of
// TW_NR row slots. Warp roles:
//   warp 0 (one lane): TMA loads of the next input row (zero-filled outside the image)
//     into the next slot once that slot is free, completing on the slot's "full" mbarrier
//     (for the image input, warps 0 and 1 build alternate rows with plain loads instead);
//   warp 2 (one lane, also the TMEM owner): for the next input row waits for its slot and,
//     if it opens an output row, for that row's accumulator block to be free; issues the
//     row's MMAs; commits them to the slot's "empty" mbarrier and, once an output row has
//     had its last input row, to that block's "full" mbarrier;
//   warps 3-6: wait for a full block, read their 32 TMEM lanes (warp w reads lanes
//     32 (w mod 4) ..), zero them, free the block, add the bias, ReLU and store.
// A row slot holds, per 8-channel group, pixels x0 - 1 .. x0 + 128 at 16 bytes each (2080
// bytes at a group stride of TW_GS = 2176): the A operand of shift dx and K step k starts
// at group 2k, pixel dx, with the next 8 channels one group along (leading byte offset)
// and the next 8 pixels 128 bytes on. The weights are stored [dx][group][dy][co][8], so
// that the B rows (dy, co) of one shift and group are consecutive.
// IO selects where the input rows come from and where the result goes:
//  * TW_NHWC: x and act_out NHWC; one box per group and row, 130 separate 16-byte pieces
//    (one per pixel), which the TMA unit moves one by one.
//  * TW_GROUPED: x and act_out [image][row][group][pixel][8 channels]; one group of one row
//    is a contiguous run, seen by the tensor map as 8-byte elements; per group and row two
//    1-D boxes, 128 pixels (2048 bytes, the largest box: 256 elements) from pixel x0 - 1
//    and the last 2 pixels (32 bytes) right behind them (both start on 128-byte
//    boundaries).
//  * TW_IMAGE (the network's first layer, CIN = 16): the input is the FP32 image and its
//    lambda, channels 0 and 1, rounded to BF16 by the loading warp, which writes them into
//    group 0 of the slot (channels 2..15 stay zero); act_out grouped.
//  * TW_HEAD (the last layer, COUT = 16): x grouped; the epilogue keeps only channel 0, o,
//    and writes p = lambda tanh(o) on the vertical edges (rows 0 .. H - 2, 0 on the last
//    row) for the dual head.
// Every wait gives up after kTcSpin polls (counted in g_tc_timeouts; the tile is then not
// written) and the other roles stop at their next wait.
constexpr int TW_NHWC = 0, TW_GROUPED = 1, TW_IMAGE = 2, TW_HEAD = 3;
// Row slots: the image rows come from plain loads, whose latency a deeper ring hides; the
// TMA rows need fewer, and a smaller ring lets four blocks share an SM.
__host__ __device__ constexpr int tw_nr(int io) { return io == TW_IMAGE ? 8 : 4; }
// TMEM accumulator blocks: 128 columns per block either way, so that four blocks fit
__host__ __device__ constexpr int tw_r(int cout) { return 128 / cout; }
constexpr int TW_THREADS = 224;     // warp 0 loads, warp 2 issues the MMAs, warps 3-6 epilogue
constexpr int TW_GS = 2176;         // bytes per 8-channel group in a row slot
constexpr int TW_ROWB = TC_P * 16;  // bytes of one group's row that the loads deliver

template <int CIN, int COUT, int IO>
constexpr size_t conv_tw_smem()
{
    // alignment slack, row slots, weights, 2 (NR + R) + 1 mbarriers, TMEM address and
    // flag, bias
    return 1024 + (size_t)tw_nr(IO) * (CIN / 8) * TW_GS + (size_t)9 * COUT * CIN * 2 +
           8 * (2 * (tw_nr(IO) + tw_r(COUT)) + 1) + 16 + 4 * COUT;
}

// Wait for the phase of parity `parity` of the mbarrier at `bar`; false (and *bad set) after
// kTcSpin polls or once another role has set *bad.
__device__ __forceinline__ bool tw_wait(unsigned bar, unsigned parity, volatile int *bad)
{
    for (unsigned it = 0; it < kTcSpin; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 1023u) == 1023u && *bad) return false;
    }
    if (atomicExch((int *)bad, 1) == 0) atomicAdd(&g_tc_timeouts, 1u);
    return false;
}

// Zero N (16 or 32) TMEM columns of the calling warp's 32 lanes from taddr.
template <int N>
__device__ __forceinline__ void tc_st_zero(unsigned taddr)
{
    static_assert(N == 16 || N == 32, "tcgen05.st of 16 or 32 columns");
    const unsigned z = 0;
    if constexpr (N == 32) {
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
            "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};\n" ::"r"(taddr),
            "r"(z)
            : "memory");
    } else {
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};\n" ::"r"(
                taddr),
            "r"(z)
            : "memory");
    }
}

// Chunk c: rows y0 .. y0 + n - 1 of the pixel column starting at x0 of image b.
struct TwChunk {
    int b, x0, y0, n;
};
__device__ __forceinline__ TwChunk tw_chunk(long long c, int cpc, int L, int tiles_x, int H)
{
    const long long col = c / cpc;
    TwChunk r;
    r.b = (int)(col / tiles_x);
    r.x0 = (int)(col % tiles_x) * TC_M;
    r.y0 = (int)(c % cpc) * L;
    r.n = min(L, H - r.y0);
    return r;
}

// Walks the input rows of a block's chunks in load order (n + 2 rows per chunk).
struct TwRows {
    long long c, nchunks;
    int r, cpc, L, tiles_x, H;
    TwChunk ch;
    __device__ __forceinline__ bool valid() const { return c < nchunks; }
    __device__ __forceinline__ void start(long long c0, long long nc, int cpc_, int L_, int tx_, int H_)
    {
        c = c0;
        nchunks = nc;
        cpc = cpc_;
        L = L_;
        tiles_x = tx_;
        H = H_;
        r = 0;
        if (c < nchunks) ch = tw_chunk(c, cpc, L, tiles_x, H);
    }
    __device__ __forceinline__ void next(long long stride)
    {
        if (++r == ch.n + 2) {
            r = 0;
            c += stride;
            if (c < nchunks) ch = tw_chunk(c, cpc, L, tiles_x, H);
        }
    }
};

// accumulator block of output row o (counted along the block's rows) in a ring of R
template <int R>
__device__ __forceinline__ int tw_block(unsigned o)
{
    return R - 1 - (int)(o % R);
}

template <int CIN, int COUT, int IO>
__global__ void __launch_bounds__(TW_THREADS, 4)
    conv3x3_tw(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmap_tail,
               int B, int H, int W, int L, const __nv_bfloat16 *Wt, const float *bias, int relu,
               float *pre_out, __nv_bfloat16 *act_out, const float *img, const float *lam, float *p_out)
{
    static_assert(IO != TW_IMAGE || CIN == 16, "the image input has 16 (2 non-zero) channels");
    static_assert(IO != TW_HEAD || COUT == 16, "the head reads a 16-channel output");
    constexpr int TW_NR = tw_nr(IO), TW_R = tw_r(COUT);
    constexpr bool GROUPED_OUT = IO == TW_GROUPED || IO == TW_IMAGE;
    constexpr int KG = CIN / 8;
    constexpr int SLOT = KG * TW_GS;
    constexpr unsigned RBYTES = KG * TW_ROWB;
    constexpr int NCOL = TW_R * COUT;  // TMEM columns (128)
    extern __shared__ __align__(1024) unsigned char smem_tw[];
    unsigned char *base = smem_tw + ((1024u - (smem_u32(smem_tw) & 1023u)) & 1023u);
    unsigned char *bbuf = base + TW_NR * SLOT;
    unsigned char *barp = bbuf + 9 * COUT * CIN * 2;
    unsigned *tslot = reinterpret_cast<unsigned *>(barp + 8 * (2 * (TW_NR + TW_R) + 1));
    volatile int *bad = reinterpret_cast<volatile int *>(tslot + 1);
    float *bias_s = reinterpret_cast<float *>(tslot + 4);
    const unsigned a_s = smem_u32(base), b_s = smem_u32(bbuf), bar0 = smem_u32(barp);
    // mbarriers: full[s], empty[s] of the row slots, full[k], empty[k] of the blocks, and
    // one that the MMA lane's last commit completes
    auto r_full = [&](int s) { return bar0 + 8u * s; };
    auto r_empty = [&](int s) { return bar0 + 8u * (TW_NR + s); };
    auto c_full = [&](int k) { return bar0 + 8u * (2 * TW_NR + k); };
    auto c_empty = [&](int k) { return bar0 + 8u * (2 * TW_NR + TW_R + k); };
    const unsigned mma_done = bar0 + 8u * (2 * TW_NR + 2 * TW_R);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = (W + TC_M - 1) / TC_M;
    const int cpc = (H + L - 1) / L;  // chunks per column
    const long long nchunks = (long long)B * tiles_x * cpc;

    if (IO == TW_IMAGE)  // channels 2..15 of the image rows stay zero
        for (int t = tid; t < TW_NR * SLOT / 16; t += TW_THREADS)
            reinterpret_cast<uint4 *>(base)[t] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int q = 0; q < TW_NR; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(r_full(q)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(r_empty(q)) : "memory");
        }
        for (int q = 0; q < TW_R; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(c_full(q)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(c_empty(q)) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mma_done) : "memory");
        *bad = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(tslot)),
                     "n"(NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    // Everything above is on chip. Launched with a programmatic dependency, the block got
    // here while the previous kernel of the stream finished; every global read (weights
    // included) comes after that kernel's completion.
    pdl_enter();
    // weights: [dx][group][dy][co][8 channels]
    for (int t = tid; t < 9 * KG * COUT; t += TW_THREADS) {
        const int co = t % COUT, dy = (t / COUT) % 3, g = (t / (3 * COUT)) % KG, dx = t / (3 * COUT * KG);
        *reinterpret_cast<uint4 *>(bbuf + (size_t)t * 16) =
            *reinterpret_cast<const uint4 *>(Wt + ((long long)co * 9 + dy * 3 + dx) * CIN + g * 8);
    }
    if (tid < COUT) bias_s[tid] = bias ? bias[tid] : 0.f;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // weights for the MMAs
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = *tslot;
    if (warp >= 3) {  // every accumulator block starts at zero
        const unsigned lanes = (unsigned)((warp & 3) * 32) << 16;
#pragma unroll
        for (int c = 0; c < NCOL; c += COUT) tc_st_zero<COUT>(tmem + lanes + (unsigned)c);
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

    if (IO == TW_IMAGE && warp < 2) {
        // warps 0 and 1 build alternate rows (load-order rows q = warp, warp + 2, ..): pixel
        // x0 - 1 + px of row y becomes (bf16 f, bf16 lambda, 0, ..); each warp loads its
        // next row into registers before it waits for a slot and stores the current one
        TwRows it;
        it.start(blockIdx.x, nchunks, cpc, L, tiles_x, H);
        if (warp == 1) it.next(gridDim.x);
        float cur[5], nxt[5];
        unsigned cmask = 0u, nmask = 0u;
        float clam = 0.f, nlam = 0.f;
        auto load_row = [&](const TwRows &rw, float (&v)[5], unsigned &mask, float &lv) {
            const int y = rw.ch.y0 - 1 + rw.r;
            const float *src = img + ((long long)rw.ch.b * H + (y < 0 ? 0 : y)) * W;
            lv = lam[rw.ch.b];
            mask = 0u;
#pragma unroll
            for (int kk = 0; kk < 5; ++kk) {
                const int x = rw.ch.x0 - 1 + lane + 32 * kk;
                const bool in = lane + 32 * kk < TC_P && y >= 0 && y < H && x >= 0 && x < W;
                v[kk] = in ? src[x] : 0.f;
                mask |= in ? 1u << kk : 0u;
            }
        };
        if (it.valid()) load_row(it, cur, cmask, clam);
        bool ok = true;
        for (unsigned q = (unsigned)warp; it.valid() && ok; q += 2u) {
            TwRows nx = it;
            nx.next(gridDim.x);
            nx.next(gridDim.x);
            if (nx.valid()) load_row(nx, nxt, nmask, nlam);
            const int sl = (int)(q % TW_NR);
            int got = 1;
            if (lane == 0) got = tw_wait(r_empty(sl), ((q / TW_NR) & 1u) ^ 1u, bad) ? 1 : 0;
            if (!__shfl_sync(0xffffffffu, got, 0)) {
                ok = false;
                break;
            }
            unsigned char *dst = base + sl * SLOT;
#pragma unroll
            for (int kk = 0; kk < 5; ++kk) {
                const int px = lane + 32 * kk;
                if (px < TC_P) {
                    unsigned v = 0u;
                    if (cmask >> kk & 1u) {
                        const __nv_bfloat162 h = __floats2bfloat162_rn(cur[kk], clam);
                        v = *reinterpret_cast<const unsigned *>(&h);
                    }
                    *reinterpret_cast<unsigned *>(dst + px * 16) = v;
                }
            }
            // the generic-proxy writes become visible to the MMAs (async proxy)
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(r_full(sl)) : "memory");
            it = nx;
#pragma unroll
            for (int kk = 0; kk < 5; ++kk) cur[kk] = nxt[kk];
            cmask = nmask;
            clam = nlam;
        }
    } else if (warp == 0) {
        if (lane == 0) {
            long long q = 0;  // rows issued by this block
            int sl = 0;       // its slot (q mod TW_NR) and the parity of that slot's fill
            unsigned lp = 0;
            bool ok = true;
            for (long long c = blockIdx.x; c < nchunks && ok; c += gridDim.x) {
                const TwChunk ch = tw_chunk(c, cpc, L, tiles_x, H);
                for (int r = 0; r < ch.n + 2; ++r) {
                    if (!tw_wait(r_empty(sl), lp ^ 1u, bad)) {
                        ok = false;
                        break;
                    }
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(r_full(sl)),
                                 "r"(RBYTES)
                                 : "memory");
                    const int y = ch.y0 - 1 + r;
                    const unsigned d0 = a_s + sl * SLOT;
#pragma unroll
                    for (int g = 0; g < KG; ++g) {
                        if constexpr (IO != TW_NHWC) {
                            // 8-byte elements: pixel p of a row starts at element 2 p
                            asm volatile(
                                "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
                                " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(d0 + g * TW_GS),
                                "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(2 * (ch.x0 - 1)), "r"(g), "r"(y),
                                "r"(ch.b), "r"(r_full(sl))
                                : "memory");
                            asm volatile(
                                "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
                                " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(d0 + g * TW_GS + 2048),
                                "l"(reinterpret_cast<uint64_t>(&tmap_tail)), "r"(2 * (ch.x0 + 127)), "r"(g),
                                "r"(y), "r"(ch.b), "r"(r_full(sl))
                                : "memory");
                        } else {
                            asm volatile(
                                "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
                                " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(d0 + g * TW_GS),
                                "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(0), "r"(g), "r"(ch.x0 - 1),
                                "r"(y), "r"(ch.b), "r"(r_full(sl))
                                : "memory");
                        }
                    }
                    ++q;
                    if (++sl == TW_NR) {
                        sl = 0;
                        lp ^= 1u;
                    }
                }
            }
            // after a wait gave up: let the copies of every slot's last load land before the
            // block exits (the phase of that load completes once its bytes arrive)
            if (*bad) {
                for (int s = 0; s < TW_NR && s < q; ++s) {
                    const long long last = s + ((q - 1 - s) / TW_NR) * TW_NR;
                    const unsigned par = (unsigned)(last / TW_NR) & 1u;
                    for (unsigned it = 0; it < kTcSpin; ++it) {
                        unsigned done;
                        asm volatile(
                            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                            " selp.u32 %0, 1, 0, p;\n}\n"
                            : "=r"(done)
                            : "r"(r_full(s)), "r"(par)
                            : "memory");
                        if (done) break;
                    }
                }
            }
        }
    } else if (warp == 2) {
        if (lane == 0) {
            // The issuing lane runs alone, so its scalar work is on the critical path: slots,
            // blocks and parities advance as counters, and each descriptor is a base
            // descriptor plus an offset (the start address >> 4 lives in the low 14 bits and
            // shared addresses stay below 256 KB, so the add cannot carry out of it).
            constexpr uint32_t idesc0 = tc_idesc(TC_M, 16) & ~(0x3Fu << 17);  // N set per MMA
            const uint64_t a0d = tc_desc(a_s, TW_GS, 128), b0d = tc_desc(b_s, 3 * COUT * 16, 128);
            int sl = 0;       // slot of the next input row and the parity of its fill
            unsigned sp = 0;
            unsigned o0 = 0;  // output rows of the finished chunks
            bool ok = true;
            for (long long c = blockIdx.x; c < nchunks && ok; c += gridDim.x) {
                const TwChunk ch = tw_chunk(c, cpc, L, tiles_x, H);
                for (int i = 0; i < ch.n + 2; ++i) {
                    // input row i of the chunk feeds its output rows i - dy, dy = dlo .. dhi
                    ok = tw_wait(r_full(sl), sp, bad);
                    if (ok && i < ch.n) {  // opens output row i: its block must be free
                        const unsigned o = o0 + (unsigned)i;
                        ok = tw_wait(c_empty(tw_block<TW_R>(o)), ((o / TW_R) & 1u) ^ 1u, bad);
                    }
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const int dlo = max(0, i - (ch.n - 1)), dhi = min(2, i);
                    const int nb = dhi - dlo + 1;
                    const int k0 = tw_block<TW_R>(o0 + (unsigned)(i - dlo));  // block of the lowest column
                    const int m = min(nb, TW_R - k0);                    // blocks before the wrap
                    const unsigned acc1 = tmem + (unsigned)(k0 * COUT), acc2 = tmem;
                    const uint32_t id1 = idesc0 | ((uint32_t)(m * COUT) >> 3) << 17;
                    const uint32_t id2 = idesc0 | ((uint32_t)((nb - m) * COUT) >> 3) << 17;
                    const uint64_t ar = a0d + (uint64_t)(sl * (SLOT >> 4));
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
                        for (int ks = 0; ks < KG / 2; ++ks) {
                            const uint64_t ad = ar + (uint64_t)((2 * ks * TW_GS + dx * 16) >> 4);
                            // B rows (dy, co) of this shift and K step, from dy = dlo
                            const uint64_t bd = b0d + (uint64_t)(((dx * KG + 2 * ks) * 3 + dlo) * COUT);
                            asm volatile(
                                "{\n .reg .pred p;\n setp.eq.u32 p, 1, 1;\n"
                                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc1),
                                "l"(ad), "l"(bd), "r"(id1)
                                : "memory");
                            if (m < nb)
                                asm volatile(
                                    "{\n .reg .pred p;\n setp.eq.u32 p, 1, 1;\n"
                                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc2),
                                    "l"(ad), "l"(bd + (uint64_t)(m * COUT)), "r"(id2)
                                    : "memory");
                        }
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                            r_empty(sl))
                        : "memory");
                    if (i >= 2)  // output row i - 2 has had its last input row
                        asm volatile(
                            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                c_full(tw_block<TW_R>(o0 + (unsigned)(i - 2))))
                            : "memory");
                    if (++sl == TW_NR) {
                        sl = 0;
                        sp ^= 1u;
                    }
                }
                o0 += (unsigned)ch.n;
            }
            // every MMA issued completes before the accumulators are released
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mma_done)
                : "memory");
            for (unsigned it = 0; it < kTcSpin; ++it) {
                unsigned done;
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                    " selp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(done)
                    : "r"(mma_done), "r"(0u)
                    : "memory");
                if (done) break;
            }
        }
    } else if (warp >= 3) {
        const int lg = warp & 3;  // TMEM lanes 32 lg .. 32 lg + 31 (pixels of the tile)
        const unsigned lanes = (unsigned)(lg * 32) << 16;
        unsigned o = 0;
        bool ok = true;
        for (long long ck = blockIdx.x; ck < nchunks && ok; ck += gridDim.x) {
            const TwChunk ch = tw_chunk(ck, cpc, L, tiles_x, H);
            for (int j = 0; j < ch.n; ++j, ++o) {
                const int k = tw_block<TW_R>(o);
                int got = 1;
                if (lane == 0) got = tw_wait(c_full(k), (o / TW_R) & 1u, bad) ? 1 : 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                float v[COUT];
                const unsigned ta = tmem + lanes + (unsigned)(k * COUT);
                tc_ld<COUT>(ta, v);
                tc_st_zero<COUT>(ta);
                asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(c_empty(k)) : "memory");
                const long long row = (long long)ch.b * H + ch.y0 + j;
                const int x = ch.x0 + lg * 32 + lane;
                if (IO == TW_HEAD && x < W) {
                    p_out[row * W + x] = ch.y0 + j < H - 1 ? lam[ch.b] * tanhf(v[0] + bias_s[0]) : 0.f;
                } else if (x < W) {
                    const long long pbase = (row * W + x) * COUT;
#pragma unroll
                    for (int c = 0; c < COUT; c += 8) {
                        float q[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) q[e] = v[c + e] + bias_s[c + e];
                        if (pre_out) {
                            *reinterpret_cast<float4 *>(pre_out + pbase + c) = make_float4(q[0], q[1], q[2], q[3]);
                            *reinterpret_cast<float4 *>(pre_out + pbase + c + 4) = make_float4(q[4], q[5], q[6], q[7]);
                        }
                        if (act_out) {
                            unsigned u[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                float a0 = q[2 * e], a1 = q[2 * e + 1];
                                if (relu) {
                                    a0 = fmaxf(a0, 0.f);
                                    a1 = fmaxf(a1, 0.f);
                                }
                                const __nv_bfloat162 h = __floats2bfloat162_rn(a0, a1);
                                u[e] = *reinterpret_cast<const unsigned *>(&h);
                            }
                            // NHWC, or grouped: [image][row][8-channel group][pixel][8]
                            const long long o8 = GROUPED_OUT ? ((row * (COUT / 8) + c / 8) * W + x) * 8 : pbase + c;
                            *reinterpret_cast<uint4 *>(act_out + o8) = make_uint4(u[0], u[1], u[2], u[3]);
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 2)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(NCOL) : "memory");
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to the driver library)
typedef CUresult (*TmapEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

TmapEncodeFn tmap_encoder()
{
    static TmapEncodeFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            (void)cudaGetLastError();
            return (TmapEncodeFn) nullptr;
        }
        return (TmapEncodeFn)f;
    }();
    return fn;
}

template <int CIN, int COUT, int IO>
tv_status launch_conv_tw(const __nv_bfloat16 *X, int B, int H, int W, const __nv_bfloat16 *Wt,
                         const float *bias, int relu, float *pre_out, __nv_bfloat16 *act_out,
                         cudaStream_t s, const float *img = nullptr, const float *lam = nullptr,
                         float *p_out = nullptr)
{
    TmapEncodeFn enc = tmap_encoder();
    if (!enc) {
        set_error("tv_net_conv3x3: cuTensorMapEncodeTiled is not available from the driver");
        return TV_ERR_CUDA;
    }
    // NHWC: the activation as a 5-D BF16 tensor, 8 channels x CIN/8 groups x W x H x B, one
    // box per group and row (8 x 1 x 130 pixels x 1 x 1). Grouped: a 4-D tensor of 8-byte
    // elements, 2 W x CIN/8 groups x H x B, boxes of 256 and of 4 elements of one row.
    CUtensorMap tmap, tmap_tail;
    const cuuint64_t KG = CIN / 8;
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r0 = CUDA_SUCCESS, r1 = CUDA_SUCCESS;
    if (IO == TW_IMAGE) {
        memset(&tmap, 0, sizeof(tmap));  // not read: the rows come from the image
        tmap_tail = tmap;
    } else if (IO != TW_NHWC) {
        const cuuint64_t dims[4] = {2 * (cuuint64_t)W, KG, (cuuint64_t)H, (cuuint64_t)B};
        const cuuint64_t strides[3] = {(cuuint64_t)W * 16, (cuuint64_t)W * CIN * 2,
                                       (cuuint64_t)H * W * CIN * 2};
        const cuuint32_t box[4] = {256, 1, 1, 1}, box_tail[4] = {4, 1, 1, 1};
        r0 = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<__nv_bfloat16 *>(X), dims, strides, box,
                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        r1 = enc(&tmap_tail, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<__nv_bfloat16 *>(X), dims, strides,
                 box_tail, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        const cuuint64_t dims[5] = {8, KG, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
        const cuuint64_t strides[4] = {16, 16 * KG, (cuuint64_t)W * CIN * 2, (cuuint64_t)H * W * CIN * 2};
        const cuuint32_t box[5] = {8, 1, (cuuint32_t)TC_P, 1, 1};
        r0 = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16 *>(X), dims, strides, box,
                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        tmap_tail = tmap;  // not read
    }
    if (r0 != CUDA_SUCCESS || r1 != CUDA_SUCCESS) {
        set_error("tv_net_conv3x3: cuTensorMapEncodeTiled rejected the activation layout");
        return TV_ERR_INVALID;
    }
    auto kern = conv3x3_tw<CIN, COUT, IO>;
    constexpr size_t smem = conv_tw_smem<CIN, COUT, IO>();
    static bool attr = false;
    if (!attr) {
        tv_status st0 = check_cuda(
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
            "cudaFuncSetAttribute");
        if (st0 != TV_OK) return st0;
        st0 = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                              (int)cudaSharedmemCarveoutMaxShared),
                         "cudaFuncSetAttribute");
        if (st0 != TV_OK) return st0;
        attr = true;
    }
    // resident blocks per SM from registers, shared memory and TMEM columns (the occupancy
    // query reports one block for a kernel that allocates TMEM, whatever it allocates)
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaFuncAttributes fa;
        int dev = 0, smem_sm = 0, regs_sm = 0;
        tv_status st0 = check_cuda(cudaFuncGetAttributes(&fa, kern), "cudaFuncGetAttributes");
        if (st0 == TV_OK) st0 = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
        if (st0 == TV_OK)
            st0 = check_cuda(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev),
                             "cudaDeviceGetAttribute");
        if (st0 == TV_OK)
            st0 = check_cuda(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev),
                             "cudaDeviceGetAttribute");
        if (st0 != TV_OK) return st0;
        const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;  // allocated per warp
        const int by_regs = regs_sm / (warp_regs * (TW_THREADS / 32));
        const int by_smem = smem_sm / (int)(smem + 1024);         // 1 KB reserved per block
        per_sm = std::max(1, std::min(std::min(by_regs, by_smem), 512 / (tw_r(COUT) * COUT)));
    }
    // chunks of L rows: about one per block, each loading L + 2 input rows for L tiles
    const long long cols = (long long)B * ((W + TC_M - 1) / TC_M);
    const long long slots = (long long)per_sm * sm_count_current();
    const long long L = std::max(1LL, std::min<long long>(H, (cols * H + slots - 1) / slots));
    const long long nchunks = cols * ((H + L - 1) / L);
    const long long blocks = std::min(nchunks, slots);
    // with a programmatic dependency on the previous kernel (tv_set_programmatic_launch):
    // the block set-up above the kernel's pdl_enter overlaps that kernel's end
    PdlScope pdl(true);
    tv_status st = check_cuda(launch_k(kern, dim3((unsigned)blocks), dim3(TW_THREADS), smem, s, tmap,
                                       tmap_tail, B, H, W, (int)L, Wt, bias, relu, pre_out, act_out,
                                       img, lam, p_out),
                              "conv launch");
    if (st == TV_OK) note_launch();
    return st;
}

static std::atomic<int> g_net_tc{0};  // mma.sync by default: faster for N = 16/32 (see tv.h)

template <int CIN, int COUT>
tv_status launch_conv_tc(const __nv_bfloat16 *X, int B, int H, int W, const __nv_bfloat16 *Wt,
                         const float *bias, int relu, float *pre_out, __nv_bfloat16 *act_out,
                         cudaStream_t s)
{
    auto kern = conv3x3_tc<CIN, COUT>;
    constexpr size_t smem = conv_tc_smem<CIN, COUT>();
    static int per_sm = 0;
    if (per_sm == 0) {
        tv_status st0 = check_cuda(
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
            "cudaFuncSetAttribute");
        if (st0 != TV_OK) return st0;
        // the whole unified memory as shared memory, so that several blocks fit per SM
        st0 = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                              (int)cudaSharedmemCarveoutMaxShared),
                         "cudaFuncSetAttribute");
        if (st0 != TV_OK) return st0;
        // blocks per SM from the shared memory (the occupancy query does not see that
        // a block holds only 64 of the 512 TMEM columns); at most 4, 256 columns
        const int b = (int)((227 * 1024) / (smem + 1024));
        per_sm = b < 1 ? 1 : (b > 4 ? 4 : b);
    }
    const long long ntiles = (long long)B * H * ((W + TC_M - 1) / TC_M);
    long long blocks = (long long)per_sm * sm_count_current();
    if (blocks > ntiles) blocks = ntiles;
    kern<<<(unsigned)blocks, NTHR, smem, s>>>(X, B, H, W, Wt, bias, relu, pre_out, act_out);
    tv_status st = check_cuda(cudaGetLastError(), "conv launch");
    if (st == TV_OK) note_launch();
    return st;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

// grid.y = ceil(H / TH) and grid.z = B are limited to 65535
bool valid_shape(int B, int H, int W)
{
    return B >= 1 && H >= 1 && W >= 1 && B <= 65535 && (H + TH - 1) / TH <= 65535;
}

__global__ void cast_bf16(const float *a, long long n, __nv_bfloat16 *out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16(a[i]);
}


// ---------------------------------------------------------------- inference --
// The first layer of the network specialised for inference, on the CUDA cores.
constexpr int FT = 16;  // 16 x 16 output pixels per block, 256 threads

// Layer 1: the packed input has two non-zero channels, the image and lambda, both rounded
// to BF16 and zero outside the image, so
//     out[co] = bias[co] + sum over the taps inside the image of w[co][tap][0] f + w[co][tap][1] lambda,
// then ReLU and BF16 (32 channels). The products of BF16 values are exact in FP32 and are
// summed in FP32, as on the tensor cores (in another order); no packed input is written.
// 128 threads per 16 x 16 tile, two pixels (rows ty and ty + 8) per thread, so that each
// weight read from shared memory serves both.
__device__ __forceinline__ void store_act32(__nv_bfloat16 *dst, const float (&acc)[32])
{
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        unsigned u[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(acc[q * 8 + 2 * e], 0.f),
                                                           fmaxf(acc[q * 8 + 2 * e + 1], 0.f));
            u[e] = *reinterpret_cast<const unsigned *>(&h);
        }
        d[q] = make_uint4(u[0], u[1], u[2], u[3]);
    }
}

// the same, into the grouped layout: group q of this pixel at dst + q * W * 8
__device__ __forceinline__ void store_act32_grouped(__nv_bfloat16 *dst, int W, const float (&acc)[32])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        unsigned u[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(acc[q * 8 + 2 * e], 0.f),
                                                           fmaxf(acc[q * 8 + 2 * e + 1], 0.f));
            u[e] = *reinterpret_cast<const unsigned *>(&h);
        }
        *reinterpret_cast<uint4 *>(dst + (long long)q * W * 8) = make_uint4(u[0], u[1], u[2], u[3]);
    }
}

__global__ void __launch_bounds__(128)
    first_layer(const float *f, int H, int W, const float *lam, const __nv_bfloat16 *Wt,
                const float *bias, __nv_bfloat16 *act, bool grouped)
{
    __shared__ __align__(16) float wsm[9][2][32];  // [tap][image, lambda][co]
    __shared__ __align__(16) float bsm[32];
    __shared__ float patch[FT + 2][FT + 2];
    const int b = blockIdx.z;
    const int x0 = blockIdx.x * FT, y0 = blockIdx.y * FT;
    for (int t = threadIdx.x; t < 9 * 2 * 32; t += blockDim.x) {
        const int co = t & 31, ch = (t >> 5) & 1, tap = t >> 6;
        wsm[tap][ch][co] = __bfloat162float(Wt[(co * 9 + tap) * 16 + ch]);
    }
    if (threadIdx.x < 32) bsm[threadIdx.x] = bias ? bias[threadIdx.x] : 0.f;
    const float *fb = f + (long long)b * H * W;
    for (int t = threadIdx.x; t < (FT + 2) * (FT + 2); t += blockDim.x) {
        const int py = t / (FT + 2), px = t % (FT + 2);
        const int gy = y0 + py - 1, gx = x0 + px - 1;
        float v = 0.f;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W)
            v = __bfloat162float(__float2bfloat16(fb[(long long)gy * W + gx]));
        patch[py][px] = v;
    }
    __syncthreads();
    const int ty = threadIdx.x / FT, tx = threadIdx.x % FT;  // rows ty and ty + 8
    const int x = x0 + tx, ya = y0 + ty, yb = ya + 8;
    if (x >= W || ya >= H) return;
    const float lb = __bfloat162float(__float2bfloat16(lam[b]));
    float acc0[32], acc1[32];
#pragma unroll
    for (int co = 0; co < 32; ++co) acc0[co] = acc1[co] = bsm[co];
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
        const int gx = x + kx - 1;
        const bool inx = gx >= 0 && gx < W;
        const int ga = ya + ky - 1, gb = yb + ky - 1;
        const float va = patch[ty + ky][tx + kx], vb = patch[ty + 8 + ky][tx + kx];
        const float la = (inx && ga >= 0 && ga < H) ? lb : 0.f;
        const float lbb = (inx && gb >= 0 && gb < H) ? lb : 0.f;
        const float4 *w0 = reinterpret_cast<const float4 *>(&wsm[tap][0][0]);
        const float4 *w1 = reinterpret_cast<const float4 *>(&wsm[tap][1][0]);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 a = w0[q], c = w1[q];
            acc0[4 * q + 0] = fmaf(a.x, va, fmaf(c.x, la, acc0[4 * q + 0]));
            acc0[4 * q + 1] = fmaf(a.y, va, fmaf(c.y, la, acc0[4 * q + 1]));
            acc0[4 * q + 2] = fmaf(a.z, va, fmaf(c.z, la, acc0[4 * q + 2]));
            acc0[4 * q + 3] = fmaf(a.w, va, fmaf(c.w, la, acc0[4 * q + 3]));
            acc1[4 * q + 0] = fmaf(a.x, vb, fmaf(c.x, lbb, acc1[4 * q + 0]));
            acc1[4 * q + 1] = fmaf(a.y, vb, fmaf(c.y, lbb, acc1[4 * q + 1]));
            acc1[4 * q + 2] = fmaf(a.z, vb, fmaf(c.z, lbb, acc1[4 * q + 2]));
            acc1[4 * q + 3] = fmaf(a.w, vb, fmaf(c.w, lbb, acc1[4 * q + 3]));
        }
    }
    if (grouped) {
        store_act32_grouped(act + ((long long)b * H + ya) * 4 * W * 8 + (long long)x * 8, W, acc0);
        if (yb < H) store_act32_grouped(act + ((long long)b * H + yb) * 4 * W * 8 + (long long)x * 8, W, acc1);
    } else {
        store_act32(act + (((long long)b * H + ya) * W + x) * 32, acc0);
        if (yb < H) store_act32(act + (((long long)b * H + yb) * W + x) * 32, acc1);
    }
}

}  // namespace

extern "C" {

int64_t tv_net_tensor_timeouts(void)
{
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_timeouts, sizeof(v)) != cudaSuccess) {
        (void)cudaGetLastError();
        return -1;
    }
    return (int64_t)v;
}

tv_status tv_net_set_tensor_path(int mode)
{
    clear_error();
    if (mode < 0 || mode > 2) {
        set_error("tv_net_set_tensor_path: 0 (mma.sync), 1 (tcgen05) or 2 (tcgen05 fed by TMA, warp roles)");
        return TV_ERR_INVALID;
    }
    g_net_tc.store(mode);
    return TV_OK;
}

tv_status tv_net_conv3x3(const void *d_x, int B, int H, int W, int cin, const void *d_w,
                         const float *d_bias, int cout, int relu, float *d_pre_out,
                         void *d_act_out, tv_stream_t stream)
{
    clear_error();
    if (!d_x || !d_w || (!d_act_out && !d_pre_out) || !valid_shape(B, H, W) ||
        !valid_channels(cin, cout)) {
        set_error("tv_net_conv3x3: need x, w, an output, 1 <= B <= 65535, H, W >= 1 and "
                  "channels in {16, 32}");
        return TV_ERR_INVALID;
    }
    if (!aligned16(d_x) || !aligned16(d_w) || !aligned16(d_act_out) || !aligned16(d_pre_out)) {
        set_error("tv_net_conv3x3: x, w and outputs must be 16-byte aligned");
        return TV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    auto X = static_cast<const __nv_bfloat16 *>(d_x);
    auto Wt = static_cast<const __nv_bfloat16 *>(d_w);
    auto A = static_cast<__nv_bfloat16 *>(d_act_out);
    if (g_net_tc.load() == 2) {
        if (cin == 16 && cout == 32) return launch_conv_tw<16, 32, TW_NHWC>(X, B, H, W, Wt, d_bias, relu, d_pre_out, A, s);
        if (cin == 32 && cout == 32) return launch_conv_tw<32, 32, TW_NHWC>(X, B, H, W, Wt, d_bias, relu, d_pre_out, A, s);
        if (cin == 32 && cout == 16) return launch_conv_tw<32, 16, TW_NHWC>(X, B, H, W, Wt, d_bias, relu, d_pre_out, A, s);
        return launch_conv_tw<16, 16, TW_NHWC>(X, B, H, W, Wt, d_bias, relu, d_pre_out, A, s);
    }
    if (g_net_tc.load() == 1) {
        if (cin == 16 && cout == 32) return launch_conv_tc<16, 32>(X, B, H, W, Wt, d_bias, relu, d_pre_out, A, s);
        if (cin == 32 && cout == 32) return launch_conv_tc<32, 32>(X, B, H, W, Wt, d_bias, relu, d_pre_out, A, s);
        if (cin == 32 && cout == 16) return launch_conv_tc<32, 16>(X, B, H, W, Wt, d_bias, relu, d_pre_out, A, s);
        return launch_conv_tc<16, 16>(X, B, H, W, Wt, d_bias, relu, d_pre_out, A, s);
    }
    if (cin == 16 && cout == 32) return launch_conv<16, 32, 0>(X, B, H, W, Wt, d_bias, relu, nullptr, d_pre_out, A, s);
    if (cin == 32 && cout == 32) return launch_conv<32, 32, 0>(X, B, H, W, Wt, d_bias, relu, nullptr, d_pre_out, A, s);
    if (cin == 32 && cout == 16) return launch_conv<32, 16, 0>(X, B, H, W, Wt, d_bias, relu, nullptr, d_pre_out, A, s);
    return launch_conv<16, 16, 0>(X, B, H, W, Wt, d_bias, relu, nullptr, d_pre_out, A, s);
}

tv_status tv_net_conv3x3_grouped(const void *d_x, int B, int H, int W, int cin, const void *d_w,
                                 const float *d_bias, int cout, int relu, float *d_pre_out,
                                 void *d_act_out, tv_stream_t stream)
{
    clear_error();
    if (!d_x || !d_w || (!d_act_out && !d_pre_out) || !valid_shape(B, H, W) ||
        !valid_channels(cin, cout)) {
        set_error("tv_net_conv3x3_grouped: need x, w, an output, 1 <= B <= 65535, H, W >= 1 and "
                  "channels in {16, 32}");
        return TV_ERR_INVALID;
    }
    if (!aligned16(d_x) || !aligned16(d_w) || !aligned16(d_act_out) || !aligned16(d_pre_out)) {
        set_error("tv_net_conv3x3_grouped: x, w and outputs must be 16-byte aligned");
        return TV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    auto X = static_cast<const __nv_bfloat16 *>(d_x);
    auto Wt = static_cast<const __nv_bfloat16 *>(d_w);
    auto A = static_cast<__nv_bfloat16 *>(d_act_out);
    if (cin == 16 && cout == 32) return launch_conv_tw<16, 32, TW_GROUPED>(X, B, H, W, Wt, d_bias, relu, d_pre_out, A, s);
    if (cin == 32 && cout == 32) return launch_conv_tw<32, 32, TW_GROUPED>(X, B, H, W, Wt, d_bias, relu, d_pre_out, A, s);
    if (cin == 32 && cout == 16) return launch_conv_tw<32, 16, TW_GROUPED>(X, B, H, W, Wt, d_bias, relu, d_pre_out, A, s);
    return launch_conv_tw<16, 16, TW_GROUPED>(X, B, H, W, Wt, d_bias, relu, d_pre_out, A, s);
}

tv_status tv_net_conv3x3_backward_data(const void *d_dy, int B, int H, int W, int cout,
                                       const void *d_w, int cin, const float *d_mask_pre,
                                       void *d_dx, void *d_scratch_w, tv_stream_t stream)
{
    clear_error();
    if (!d_dy || !d_w || !d_mask_pre || !d_dx || !d_scratch_w || !valid_shape(B, H, W) ||
        !valid_channels(cin, cout) || !aligned16(d_dy) || !aligned16(d_scratch_w) ||
        !aligned16(d_mask_pre) || !aligned16(d_dx)) {
        set_error("tv_net_conv3x3_backward_data: bad arguments (null, shape, channels or "
                  "alignment)");
        return TV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    auto Wf = static_cast<__nv_bfloat16 *>(d_scratch_w);
    flip_weights<<<ew_blocks(cin * 9 * cout), 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(d_w),
                                                           cin, cout, Wf);
    tv_status st = check_cuda(cudaGetLastError(), "flip weights");
    if (st != TV_OK) return st;
    note_launch();
    auto dY = static_cast<const __nv_bfloat16 *>(d_dy);
    auto dX = static_cast<__nv_bfloat16 *>(d_dx);
    // the convolution of dY (cout channels) with the flipped kernel gives cin channels
    if (cout == 32 && cin == 32) return launch_conv<32, 32, 1>(dY, B, H, W, Wf, nullptr, 0, d_mask_pre, nullptr, dX, s);
    if (cout == 16 && cin == 32) return launch_conv<16, 32, 1>(dY, B, H, W, Wf, nullptr, 0, d_mask_pre, nullptr, dX, s);
    if (cout == 32 && cin == 16) return launch_conv<32, 16, 1>(dY, B, H, W, Wf, nullptr, 0, d_mask_pre, nullptr, dX, s);
    return launch_conv<16, 16, 1>(dY, B, H, W, Wf, nullptr, 0, d_mask_pre, nullptr, dX, s);
}

size_t tv_net_workspace_size(int B, int H, int W)
{
    if (!valid_shape(B, H, W)) return 0;
    const size_t wg = (size_t)wgrad_blocks(B, H, W) * (32 * 9 * 32 + 32) * sizeof(float);
    const size_t hd = (size_t)ew_blocks((long long)B * H * W) * sizeof(float);
    return std::max<size_t>(std::max(wg, hd), 256);
}

tv_status tv_net_conv3x3_backward_weight(const void *d_x, const void *d_dy, int B, int H, int W,
                                         int cin, int cout, float *d_dw, float *d_db,
                                         void *d_ws, size_t ws_bytes, tv_stream_t stream)
{
    clear_error();
    if (!d_x || !d_dy || !d_dw || !d_ws || !valid_shape(B, H, W) || !valid_channels(cin, cout) ||
        !aligned16(d_x) || !aligned16(d_dy) || !aligned16(d_ws)) {
        set_error("tv_net_conv3x3_backward_weight: bad arguments (null, shape, channels or "
                  "alignment)");
        return TV_ERR_INVALID;
    }
    if (ws_bytes < (size_t)wgrad_blocks(B, H, W) * (cout * 9 * cin + cout) * sizeof(float)) {
        set_error("tv_net_conv3x3_backward_weight: workspace smaller than tv_net_workspace_size");
        return TV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    auto X = static_cast<const __nv_bfloat16 *>(d_x);
    auto dY = static_cast<const __nv_bfloat16 *>(d_dy);
    auto P = static_cast<float *>(d_ws);
    if (cin == 16 && cout == 32) return launch_wgrad<16, 32>(X, dY, B, H, W, d_dw, d_db, P, s);
    if (cin == 32 && cout == 32) return launch_wgrad<32, 32>(X, dY, B, H, W, d_dw, d_db, P, s);
    if (cin == 32 && cout == 16) return launch_wgrad<32, 16>(X, dY, B, H, W, d_dw, d_db, P, s);
    return launch_wgrad<16, 16>(X, dY, B, H, W, d_dw, d_db, P, s);
}

tv_status tv_net_pack_input(const float *d_f, int B, int H, int W, const float *d_lam, void *d_x,
                            tv_stream_t stream)
{
    clear_error();
    if (!d_f || !d_lam || !d_x || !valid_shape(B, H, W)) {
        set_error("tv_net_pack_input: bad arguments");
        return TV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const long long HW = (long long)H * W;
    const unsigned gx = (unsigned)std::max(1, ew_blocks(HW) / B);
    pack_input<<<dim3(gx, (unsigned)B), 256, 0, s>>>(d_f, H, W, d_lam,
                                                     static_cast<__nv_bfloat16 *>(d_x),
                                                     ((uintptr_t)d_x & 15) == 0);
    tv_status st = check_cuda(cudaGetLastError(), "pack input");
    if (st == TV_OK) note_launch();
    return st;
}

tv_status tv_net_first_layer(const float *d_f, int B, int H, int W, const float *d_lam,
                             const void *d_w, const float *d_bias, void *d_act_out, int grouped,
                             tv_stream_t stream)
{
    clear_error();
    if (!d_f || !d_lam || !d_w || !d_act_out || !valid_shape(B, H, W) || !aligned16(d_act_out)) {
        set_error("tv_net_first_layer: need f, lam, w and a 16-byte aligned output, "
                  "1 <= B <= 65535, H, W >= 1");
        return TV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (grouped)  // on tcgen05: the image rows built in shared memory, 3 MMAs per row
        return launch_conv_tw<16, 32, TW_IMAGE>(nullptr, B, H, W, static_cast<const __nv_bfloat16 *>(d_w),
                                                d_bias, 1, nullptr, static_cast<__nv_bfloat16 *>(d_act_out),
                                                s, d_f, d_lam);
    const dim3 grid((W + FT - 1) / FT, (H + FT - 1) / FT, B);
    first_layer<<<grid, 128, 0, s>>>(d_f, H, W, d_lam, static_cast<const __nv_bfloat16 *>(d_w),
                                     d_bias, static_cast<__nv_bfloat16 *>(d_act_out), false);
    tv_status st = check_cuda(cudaGetLastError(), "first layer");
    if (st == TV_OK) note_launch();
    return st;
}

tv_status tv_net_conv3x3_dual_head(const void *d_x, int B, int H, int W, int cin, const void *d_w,
                                   const float *d_bias, const float *d_lam, float *d_p, float *d_y,
                                   tv_stream_t stream)
{
    clear_error();
    if (!d_x || !d_w || !d_lam || !d_p || !d_y || !valid_shape(B, H, W) || !(cin == 16 || cin == 32)) {
        set_error("tv_net_conv3x3_dual_head: need x, w, lam, p and y, 1 <= B <= 65535, H, W >= 1 "
                  "and cin in {16, 32}");
        return TV_ERR_INVALID;
    }
    if (!aligned16(d_x) || !aligned16(d_w)) {
        set_error("tv_net_conv3x3_dual_head: x and w must be 16-byte aligned");
        return TV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    auto X = static_cast<const __nv_bfloat16 *>(d_x);
    auto Wt = static_cast<const __nv_bfloat16 *>(d_w);
    tv_status st = cin == 32 ? launch_conv_tw<32, 16, TW_HEAD>(X, B, H, W, Wt, d_bias, 0, nullptr, nullptr, s,
                                                              nullptr, d_lam, d_p)
                             : launch_conv_tw<16, 16, TW_HEAD>(X, B, H, W, Wt, d_bias, 0, nullptr, nullptr, s,
                                                              nullptr, d_lam, d_p);
    if (st != TV_OK) return st;
    const long long rows = (long long)B * H;
    const dim3 hg((unsigned)((W + 255) / 256), (unsigned)std::min<long long>(rows, 65535));
    {
        PdlScope pdl(true);
        st = check_cuda(launch_k(head_from_p, hg, dim3(256), 0, s, (const float *)d_p, rows, H, W, d_y),
                        "dual head");
    }
    if (st == TV_OK) note_launch();
    return st;
}

tv_status tv_net_dual_head(const float *d_o, int B, int H, int W, const float *d_lam,
                           const float *d_target, float *d_y, float *d_loss, void *d_grad_o,
                           void *d_ws, size_t ws_bytes, tv_stream_t stream)
{
    clear_error();
    if (!d_o || !d_lam || !d_y || !valid_shape(B, H, W) || (d_grad_o && !d_target) ||
        (d_loss && !d_target)) {
        set_error("tv_net_dual_head: need o, lam, y (and a target for the loss or gradient)");
        return TV_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = (long long)B * H * W;
    const int blocks = ew_blocks(N);
    if (d_loss && (!d_ws || ws_bytes < (size_t)blocks * sizeof(float))) {
        set_error("tv_net_dual_head: the loss needs a workspace of tv_net_workspace_size bytes");
        return TV_ERR_INVALID;
    }
    const float inv = 1.f / (float)N;
    float *part = d_loss ? static_cast<float *>(d_ws) : nullptr;
    dual_head<<<blocks, 256, 0, s>>>(d_o, B, H, W, d_lam, d_target, d_y, part, inv);
    tv_status st = check_cuda(cudaGetLastError(), "dual head");
    if (st != TV_OK) return st;
    note_launch();
    if (d_loss) {
        sum_partials<<<1, 256, 0, s>>>(part, blocks, d_loss);
        st = check_cuda(cudaGetLastError(), "loss sum");
        if (st != TV_OK) return st;
        note_launch();
    }
    if (d_grad_o) {
        dual_head_grad<<<blocks, 256, 0, s>>>(d_o, B, H, W, d_lam, d_y, d_target,
                                               static_cast<__nv_bfloat16 *>(d_grad_o), inv);
        st = check_cuda(cudaGetLastError(), "dual head gradient");
        if (st == TV_OK) note_launch();
    }
    return st;
}

tv_status tv_net_adam(float *d_w, float *d_m, float *d_v, float *d_g, int64_t n, float lr,
                      float beta1, float beta2, float eps, int step, void *d_w_bf16,
                      tv_stream_t stream)
{
    clear_error();
    if (!d_w || !d_m || !d_v || !d_g || n < 0 || step < 1) {
        set_error("tv_net_adam: bad arguments");
        return TV_ERR_INVALID;
    }
    if (n == 0) return TV_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const float bc1 = 1.f - powf(beta1, (float)step), bc2 = 1.f - powf(beta2, (float)step);
    adam_step<<<ew_blocks(n), 256, 0, s>>>(d_w, d_m, d_v, d_g, n, lr, beta1, beta2, eps, bc1, bc2,
                                           static_cast<__nv_bfloat16 *>(d_w_bf16));
    tv_status st = check_cuda(cudaGetLastError(), "adam");
    if (st == TV_OK) note_launch();
    return st;
}

tv_status tv_net_cast_bf16(const float *d_a, int64_t n, void *d_out, tv_stream_t stream)
{
    clear_error();
    if (n < 0 || (n > 0 && (!d_a || !d_out))) {
        set_error("tv_net_cast_bf16: bad arguments");
        return TV_ERR_INVALID;
    }
    if (n == 0) return TV_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cast_bf16<<<ew_blocks(n), 256, 0, s>>>(d_a, n, static_cast<__nv_bfloat16 *>(d_out));
    tv_status st = check_cuda(cudaGetLastError(), "cast");
    if (st == TV_OK) note_launch();
    return st;
}

}  // extern "C"
