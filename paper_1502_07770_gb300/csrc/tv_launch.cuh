// Launch of a batch-of-chains kernel, shared by the chain and 2D entry points:
// launch shape, shared-memory opt-in, launch counting and optional per-launch
// CUDA-event timing (for benchmarks; off by default).
#pragma once
#include "tv_coop.cuh"
#include "tv_dp.cuh"
#include "tv_host.h"

namespace tvh {

enum ProfKind { PK_CHAIN = 0, PK_COL = 1, PK_ROW = 2, PK_INIT = 3, PK_GRAD = 4, PK_N = 5 };

void note_launch();
bool prof_on();
void prof_mark(int kind, cudaStream_t s, bool start);
// Timed launches of `kind` recorded and not yet read, and the removal of those from
// index `first` on (launches an entry point knows did no work, e.g. the phases of a
// 2D solve launched after its stop flag was set, which return at once).
size_t prof_pending(int kind);
void prof_drop_from(int kind, size_t first);

// Warps per block of a one-thread-per-chain launch: the spread of batch_shape for
// small batches; for batches of at least two warps per SM, the largest block (up to
// 4 warps) whose resident warps (shared memory and registers permitting) hold the
// whole batch in one wave, else the one with the most resident warps. Occupancy
// answers are cached per kernel.
Shape chains_shape(long long warps, const void *kern, size_t per_warp);

template <class P, int RING>
tv_status launch_chains(const P &p, long long nchains, float2 *rec, float *crec, float2 *spill,
                        tvk::WsHeader *hdr, cudaStream_t s, int kind)
{
    const long long warps = (nchains + tvk::WARP - 1) / tvk::WARP;
    if (warps == 0) return TV_OK;
    const size_t per_warp = sizeof(tvk::WarpSmem<P, RING>);
    auto kern = tvk::chain_batch_kernel<P, RING>;
    tv_status st = check_cuda(
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(4 * per_warp)),
        "cudaFuncSetAttribute");
    if (st != TV_OK) return st;
    const Shape sh = chains_shape(warps, (const void *)kern, per_warp);
    const bool prof = prof_on();
    if (prof) prof_mark(kind, s, true);
    kern<<<(unsigned)sh.blocks, sh.wpb * tvk::WARP, sh.wpb * per_warp, s>>>(p, rec, crec, spill, hdr);
    st = check_cuda(cudaGetLastError(), "chain kernel launch");
    if (st == TV_OK) note_launch();
    if (prof) prof_mark(kind, s, false);
    return st;
}

// Programmatic dependent launch for the kernels of one solve (tv_set_programmatic_launch,
// on by default): inside a PdlScope(true) on the calling thread, launch_k launches with
// the stream-serialization attribute, so that a kernel becomes resident while its
// predecessor finishes (the kernels begin with tvk::pdl_enter()).
bool pdl_on();
struct PdlScope {
    bool prev;
    explicit PdlScope(bool on);
    ~PdlScope();
};

template <class... KArgs, class... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     Args... args)
{
    if (!pdl_on()) {
        kern<<<grid, block, smem, s>>>(args...);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Warp-cooperative launch: one warp per chain, `wpb` warps per block. The records
// of a chain stay in shared memory when max_len <= kCoopSmemNodes.
constexpr int kCoopSmemNodes = 4096;

int coop_split();  // 0 one warp per chain, 1 two halves in one warp, 2 two warps
int thread_split();  // 1: thread-per-chain batches run a thread per chain half

template <class P>
tv_status launch_coop(const P &p, long long nchains, int max_len, float2 *rec, float *crec,
                      float2 *spill, tvk::WsHeader *hdr, cudaStream_t s, int kind, int wpb = 4)
{
    if (nchains <= 0) return TV_OK;
    // chains long enough to split: two 16-lane halves in one warp (mode 1) or two
    // warps (mode 2, coop_pair_kernel)
    int mode = max_len >= tvk::kSplitMinLen ? coop_split() : 0;
    if constexpr (tvk::has_unary_g<P>::value) {
        if (mode == 2) mode = 1;  // general chains: one warp per chain
    }
    // few chains (at most 16 per SM): one chain per block, so that the block scheduler
    // spreads the warps evenly over the SMs (4-warp blocks leave some SMs with 8 warps
    // and others with 4 when there are about 6.7 per SM)
    if (nchains <= 16LL * sm_count_current()) wpb = mode == 2 ? 2 : 1;
    const bool pair = mode == 2 && wpb % 2 == 0;
    const int cpb = pair ? wpb / 2 : wpb;  // chains per block
    const long long blocks = (nchains + cpb - 1) / cpb;
    // records in shared memory when a block's share fits in ~200 KB, else in the workspace
    const size_t xchg = mode != 0 ? cpb * sizeof(tvk::PairXchg) : 0;
    const bool fits = max_len <= kCoopSmemNodes &&
                      xchg + cpb * tvk::coop_smem_per_warp<P>(max_len) <= (size_t)200 * 1024;
    const int smem_nodes = fits ? max_len : 0;
    const size_t smem = xchg + cpb * tvk::coop_smem_per_warp<P>(smem_nodes);
    auto kern = mode == 1 ? tvk::coop_chain_kernel<P, true> : tvk::coop_chain_kernel<P, false>;
    if constexpr (!tvk::has_unary_g<P>::value) {
        if (pair) kern = tvk::coop_pair_kernel<P>;
    }
    tv_status st = check_cuda(
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
        "cudaFuncSetAttribute");
    if (st != TV_OK) return st;
    const bool prof = prof_on();
    if (prof) prof_mark(kind, s, true);
    st = check_cuda(launch_k(kern, dim3((unsigned)blocks), dim3(wpb * tvk::WARP), smem, s, p, rec,
                             crec, spill, hdr, smem_nodes),
                    "cooperative chain kernel launch");
    if (st == TV_OK) note_launch();
    if (prof) prof_mark(kind, s, false);
    return st;
}

// Batches of fewer chains than this run one warp per chain (the update of one
// chain is then latency-bound, and a warp shortens its critical path); larger
// batches run one thread per chain.
constexpr long long kCoopMaxChainsDefault = 4096;
// The same for tv_chain_solve batches that the fixed-shape thread kernel stages 16 bytes
// at a time (uniform rows of >= 64 nodes, a multiple of 4, 16-byte aligned arrays):
// measured crossover near 2048 chains at 256 and 1024 nodes.
constexpr long long kCoopMaxChainsVec = 2048;
long long coop_max_chains();  // tunable, see tv_set_coop_max_chains
bool coop_max_auto();         // no value set (the defaults above apply)

}  // namespace tvh
