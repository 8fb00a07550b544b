/*
 * tv.h -- C ABI of the GB300 (sm_103a) total-variation library.
 *
 * The library solves, in batches on one GPU,
 *   (1) TV-l2 problems on chains (eq. 1D-ROF, Sec. 6.1)
 *           x* = argmin_x  sum_i 1/2 (x_i - y_i)^2 + sum_{i<n} w_i |x_{i+1} - x_i|
 *       by the dynamic program of Algorithm 2 specialised to quadratic unaries
 *       as in Sec. 4.1 (forward messages stored as breakpoint sequences with an
 *       implicit slope, backward clip x_i = clip(x_{i+1}, lambda^-_i, lambda^+_i));
 *   (2) the 2D ROF model of Sec. 6.1 (TV-l2 denoising on a 4-connected grid) by the
 *       Lagrangian decomposition eq. rof-saddle solved with the accelerated
 *       primal-dual iteration eq. pd, whose two proximal steps are the row chains
 *       (TV_h) and the column chains (TV_v, via the Moreau identity eq. prox-tv-conj).
 *
 * Conventions shared by every entry point
 *  - Pointers named d_* are DEVICE pointers; the caller owns every buffer and the
 *    library never frees caller memory nor allocates device memory: all scratch
 *    comes from the caller's workspace, sized by the *_workspace_size queries.
 *  - Arrays are float32, C-contiguous. An edge weight w_i belongs to the edge
 *    between node i and node i+1 of a chain.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Chain calls are
 *    asynchronous and stream-ordered; tv2d_denoise returns after the solve has
 *    finished (it reads back the iteration count and the gap).
 *  - Argument errors are reported before any launch with TV_ERR_INVALID and leave
 *    every output untouched. Errors found on the device (malformed offsets) are
 *    recorded in the workspace and read back with tv_workspace_status.
 *  - A CUDA error (including a sticky one from earlier work) returns TV_ERR_CUDA.
 *  - tv_last_error() gives a message for the calling thread's last failure.
 */
#ifndef TV_GB300_TV_H
#define TV_GB300_TV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TV_OK = 0,
    TV_ERR_INVALID = 1,        /* bad argument, or malformed offsets found on the device */
    TV_ERR_CUDA = 2,           /* a CUDA runtime call or launch failed */
    TV_ERR_NOT_CONVERGED = 3,  /* tv2d_denoise stopped at max_iters above gap_tol */
    TV_ERR_TIMEOUT = 4,        /* reserved: a bounded device wait gave up */
    TV_ERR_NOMEM = 5,          /* the workspace is smaller than the size query asked for */
    TV_ERR_CAPACITY = 6        /* a message outgrew max_breakpoints (tv_chain_solve_nonconvex) */
} tv_status;

typedef void *tv_stream_t; /* cudaStream_t */

/* Message of the calling thread's last failed call ("" if none). */
const char *tv_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int tv_version(void);

/* Number of CUDA kernels this library has launched in this process (benchmark
 * accounting; the paper has no counterpart). */
int64_t tv_launch_count(void);

/*
 * Optional per-launch timing for benchmarks (the paper has no counterpart).
 * While enabled, every solver kernel launch is bracketed by two CUDA events
 * recorded on the launch's own stream. tv_profile_read(kind, ...) waits for the
 * recorded events of one kind, returns their summed duration in milliseconds and
 * the number of launches since the previous read, and resets both. Kinds:
 * 0 chain batches (tv_chain_solve, tv_chain_solve_columns), 1 the 2D column
 * (dual) phase, 2 the 2D row (primal) phase, 3 the 2D initial row solve,
 * 4 tv_chain_solve_backward.
 * Events are created on first use and reused; TV_ERR_INVALID for a bad kind.
 */
tv_status tv_profile_enable(int on);
tv_status tv_profile_read(int kind, double *total_ms, int64_t *launches);

/* ---------------------------------------------------------------- chains ---- */

/*
 * Bytes of workspace tv_chain_solve needs for `num_chains` chains of at most
 * `max_len` nodes (about 24 bytes per node of num_chains * max_len). The workspace
 * holds the per-node records lambda^-_i, lambda^+_i of the forward pass (Sec. 4.1,
 * "Backward pass", 8 bytes per node) and a reserve for message sequences that
 * outgrow on-chip storage (at most 2n+2 breakpoints of 8 bytes per chain, the
 * bound of Sec. 4.1); the reserve is touched only by chains that need it.
 */
size_t tv_chain_workspace_size(int64_t num_chains, int64_t max_len);

/*
 * Solve eq. 1D-ROF on every chain of a batch of contiguous chains.
 *   d_y        node values, chain k at d_y[off_k .. off_{k+1}-1]
 *   d_w        per-node edge weights laid out like d_y (the entry at a chain's last
 *              node is not read), or NULL: every edge then has weight `lambda`
 *   lambda     uniform edge weight (used iff d_w == NULL); must be >= 0 and finite
 *   d_offsets  num_chains+1 monotone int64 offsets on the DEVICE, or NULL: chain k
 *              then spans [k*max_len, (k+1)*max_len) (a uniform batch)
 *   max_len    upper bound on every chain length (the uniform length if d_offsets
 *              is NULL), at most 2^24 (node counts enter the message slopes as exact
 *              FP32 integers); a chain longer than this is skipped and flagged
 *   d_x        output, same layout as d_y; must not overlap d_y or d_w. Without
 *              offsets the host checks this (TV_ERR_INVALID); with offsets the host
 *              rejects x == y or x == w, and the kernel rejects any other overlap of
 *              the node ranges [off_0, off_num_chains) (no chain is solved, and
 *              tv_workspace_status reports TV_ERR_INVALID)
 * Empty chains and chains of one node (x = y) are allowed. Weights must be >= 0.
 */
tv_status tv_chain_solve(const float *d_y, const float *d_w, float lambda,
                         const int64_t *d_offsets, int64_t num_chains, int64_t max_len,
                         float *d_x, void *d_workspace, size_t workspace_bytes,
                         tv_stream_t stream);

/*
 * tv_chain_solve for callers that cannot allocate device memory (the paper has no
 * counterpart). Some callers must not call cudaMalloc: code running inside a
 * framework that has reserved the GPU's memory for its own caching allocator, and
 * latency-critical loops that cannot take the synchronisation an allocation may
 * cause. This entry point takes only inputs and outputs, with the same meaning
 * as tv_chain_solve; its scratch is a fixed 16 MiB array in device memory that
 * every GPU loading the library holds until the process exits. That bounds the
 * batch: num_chains * max_len may be at most about 690 000 nodes (the records and
 * the reserve take about 24 bytes per node); larger batches are rejected with
 * TV_ERR_INVALID before any launch. The first call on a device looks up the
 * array's device address (make it before any stream capture); the address belongs
 * to the device's current CUDA context and is looked up again when that context
 * changes (after cudaDeviceReset, say). All calls share the array: calls that
 * overlap on the GPU race and must be ordered by the caller. Whatever the batch
 * shape, this entry point runs the one-thread-per-chain kernel (tv_chain_solve
 * picks one warp per chain for small batches and middle-rooted halves for long
 * chains), so it can be slower than tv_chain_solve on the same batch. Device-side
 * errors are not readable for this entry point (it has no caller-visible
 * workspace): malformed offsets skip the affected chains, and CSR node ranges of x
 * overlapping those of y or w skip the whole batch.
 */
tv_status tv_chain_solve_noalloc(const float *d_y, const float *d_w, float lambda,
                                 const int64_t *d_offsets, int64_t num_chains, int64_t max_len,
                                 float *d_x, tv_stream_t stream);

/*
 * General convex chains: the problem of Sec. 4 with the quadratic unaries of Sec. 4.1,
 *     x* = argmin_x sum_i (a_i x_i^2 / 2 - b_i x_i) + sum_{i<n} f_i(x_{i+1} - x_i),
 *     f_i(d) = wlo_i * d for d < 0 and whi_i * d for d >= 0,
 * with a_i > 0 and wlo_i <= whi_i (TV-l2 is a = 1, b = y, wlo = -w, whi = w; whi > 0 > wlo
 * penalises jumps up and down differently; wlo = whi adds a linear term).
 *   d_a        per-node curvature, or NULL for a_i = 1
 *   d_b, d_wlo, d_whi   per-node arrays laid out like d_y of tv_chain_solve (the entries
 *              of wlo/whi at a chain's last node are not read)
 *   d_offsets, num_chains, max_len, d_x, workspace (tv_chain_workspace_size): as for
 *              tv_chain_solve
 * Every batch runs one warp per chain (rooted at the middle node for chains of 64 nodes
 * or more). Values are not validated on the device: a_i <= 0 or wlo_i > whi_i give
 * undefined results (never an out-of-bounds access).
 */
tv_status tv_chain_solve_general(const float *d_a, const float *d_b, const float *d_wlo,
                                 const float *d_whi, const int64_t *d_offsets, int64_t num_chains,
                                 int64_t max_len, float *d_x, void *d_workspace,
                                 size_t workspace_bytes, tv_stream_t stream);

/*
 * Chains with piecewise-quadratic unaries (Sec. 4.2):
 *     x* = argmin_x sum_i (a_i x_i^2 / 2 - b_i x_i + alpha_i |x_i - f_i|) + sum_{i<n} w_i |x_{i+1} - x_i|,
 * a_i > 0, alpha_i >= 0, w_i >= 0. This is the row proximal map of TV-l1 denoising
 * (alpha = 1, a = 1/tau, b = xi/tau). One warp per chain; messages of more than 32
 * breakpoints are finished by one thread from the workspace.
 *   d_a        per-node curvature, or NULL for a_i = 1
 *   d_b, d_f   per-node arrays laid out like d_y of tv_chain_solve
 *   d_alpha    per-node l1 weights, or NULL: every node has `alpha`
 *   d_w        per-node edge weights (entry at a chain's last node unused), or NULL: `lambda`
 *   d_offsets, num_chains, max_len, d_x: as for tv_chain_solve
 *   workspace  tv_chain_pq_workspace_size(num_chains, max_len) bytes
 */
size_t tv_chain_pq_workspace_size(int64_t num_chains, int64_t max_len);
tv_status tv_chain_solve_pq(const float *d_a, const float *d_b, const float *d_alpha, float alpha,
                            const float *d_f, const float *d_w, float lambda,
                            const int64_t *d_offsets, int64_t num_chains, int64_t max_len,
                            float *d_x, void *d_workspace, size_t workspace_bytes,
                            tv_stream_t stream);

/*
 * Non-convex chains (Sec. 3): continuous piecewise-linear unaries and truncated TV,
 *     x* in argmin_x sum_i f_i(x_i) + sum_{i<n} min(w_i |x_{i+1} - x_i|, C_i),
 * solved exactly (up to FP32 rounding) by dynamic programming on the chain (eq.
 * Message:update) with piecewise-linear messages; the min-convolution with min(w|.|, C)
 * is taken as the three consecutive ones of Prop. ConsecutiveMinConvolution (Algorithm 1,
 * its mirror image, and the truncation). Each chain is rooted at its middle node and its
 * two halves run on two warps; messages of up to max_breakpoints points in shared
 * memory; every M^_i kept in the workspace for the backward pass. A minimiser need not
 * be unique: x is one of them.
 *   unaries    either CSR: d_uoff (num_nodes + 1 absolute offsets, non-decreasing), d_ulam
 *              (strictly increasing breakpoints per node) and d_uval (values there); or a
 *              grid (d_uoff = d_ulam = NULL): breakpoints 0, 1, ..., grid_len - 1 and values
 *              d_uval[i * grid_len + l] (a cost volume). A node with no breakpoint is 0.
 *   d_sl, d_sr per-node slopes of the unaries left of the first and right of the last
 *              breakpoint (NULL: the scalars sl <= 0 and sr >= 0 for every node)
 *   d_w, d_C   per-node edge weight and truncation of the edge to the next node (entry at
 *              a chain's last node unused), or NULL: the scalars w >= 0 and C >= 0 (C =
 *              INFINITY: plain TV)
 *   d_offsets, num_chains, max_len: as for tv_chain_solve (NULL offsets: num_chains
 *              chains of max_len nodes, num_nodes = num_chains * max_len)
 *   max_breakpoints  points a message may hold (1..4096; a node's breakpoint count plus
 *              the incoming message's must fit)
 *   d_x        num_nodes outputs; d_energy: num_chains optimum energies (FP64 sum of FP32
 *              message minima)
 *   workspace  tv_chain_nonconvex_workspace_size(num_nodes, num_chains, max_len,
 *              max_breakpoints) bytes (num_chains * (max_len + 1) * max_breakpoints * 8
 *              + ...).
 * A chain whose message outgrows max_breakpoints gets NaN in x and energy and the
 * workspace error word reports TV_ERR_CAPACITY (tv_workspace_status). Unaries must be
 * bounded below (sl <= 0 <= sr); other values give undefined results, never an
 * out-of-bounds access. Asynchronous on `stream`.
 */
size_t tv_chain_nonconvex_workspace_size(int64_t num_nodes, int64_t num_chains, int64_t max_len,
                                         int max_breakpoints);
tv_status tv_chain_solve_nonconvex(const int64_t *d_uoff, const float *d_ulam,
                                   const float *d_uval, int grid_len, const float *d_sl,
                                   const float *d_sr, float sl, float sr, const float *d_w,
                                   float w, const float *d_C, float C, const int64_t *d_offsets,
                                   int64_t num_nodes, int64_t num_chains, int64_t max_len,
                                   int max_breakpoints, float *d_x, double *d_energy,
                                   void *d_workspace, size_t workspace_bytes, tv_stream_t stream);

/*
 * Backward of the chain prox (vector-Jacobian product), for a differentiable TV
 * layer. From the optimality conditions of eq. 1D-ROF, on every maximal run S of
 * equal values of the solution x ("segment"), x_S = mean(y_S) + (u_r - u_{l-1})/|S|
 * with u_e = w_e sign(x_{e+1} - x_e) at the jump edges bounding S. Hence
 *     grad_y_j = mean of grad_x over the segment containing j,
 *     grad_w_e = sign(x_{e+1} - x_e) (mean_left - mean_right) at a jump edge e, and 0
 *                on edges inside a segment (grad of a uniform lambda = sum of grad_w).
 *   d_x        the solution returned by tv_chain_solve (segments are read off it:
 *              fused neighbours are bitwise equal)
 *   d_grad_x   upstream gradient, same layout
 *   d_offsets, num_chains, max_len   as for tv_chain_solve
 *   d_grad_y   output, same layout; d_grad_w optional output, same layout (the
 *              entry at a chain's last node is not written)
 *   workspace  at least 64 bytes (a device error word, read by tv_workspace_status)
 * Outputs must not alias the inputs. The derivative is the one of the solution map
 * away from degenerate points (where a jump of x is exactly zero).
 */
tv_status tv_chain_solve_backward(const float *d_x, const float *d_grad_x,
                                  const int64_t *d_offsets, int64_t num_chains, int64_t max_len,
                                  float *d_grad_y, float *d_grad_w, void *d_workspace,
                                  size_t workspace_bytes, tv_stream_t stream);

/* Bytes of workspace tv_chain_solve_columns needs for an H x W array. */
size_t tv_columns_workspace_size(int64_t H, int64_t W);

/*
 * Solve eq. 1D-ROF on the W column chains of an H x W row-major array with
 * leading dimension ld >= W (node i of column c at d_y[i*ld + c]). These are the
 * chains of the TV_v proximal step of Sec. 6.1.
 *   d_w   per-node edge weights in the same layout (row H-1 is not read), or NULL
 *   d_x   output in the same layout; must not overlap d_y or d_w
 */
tv_status tv_chain_solve_columns(const float *d_y, const float *d_w, float lambda, int64_t H,
                                 int64_t W, int64_t ld, float *d_x, void *d_workspace,
                                 size_t workspace_bytes, tv_stream_t stream);

/*
 * Read back and clear the device-side error word of a workspace used by the chain
 * calls above (synchronises `stream`). *d_status_out receives TV_OK,
 * TV_ERR_INVALID (a chain longer than max_len, or decreasing offsets) or
 * TV_ERR_CAPACITY (tv_chain_solve_nonconvex: a message outgrew max_breakpoints). When
 * overflowed != NULL it receives how many chains outgrew on-chip message storage
 * and were finished from the workspace reserve (a performance counter).
 */
tv_status tv_workspace_status(void *d_workspace, tv_stream_t stream, int *status_out,
                              int64_t *overflowed);

/* ------------------------------------------------------------------- 2D ---- */

/* Bytes of workspace tv2d_denoise needs for an H x W image and max_iters iterations. */
size_t tv2d_workspace_size(int64_t H, int64_t W, int max_iters);

/*
 * 2D TV-l2 (ROF) denoising, Sec. 6.1:
 *     x* = argmin_x 1/2 ||x - img||^2 + TV_h(x) + TV_v(x)
 * solved by the accelerated primal-dual iteration eq. pd with tau_0 = sigma_0 = 1,
 * gamma = 1, x^0 the row-chain solution at img - y^0, and the stopping rule
 * G_k / (H W) <= gap_tol on the primal-dual gap G_k of (x^{k+1}, the dual fields
 * certified by the two chain steps).
 *   d_img     H x W row-major image
 *   d_wh      H x (W-1) horizontal edge weights (edge (r,c)-(r,c+1) at r*(W-1)+c), or NULL
 *   d_wv      (H-1) x W vertical edge weights (edge (r,c)-(r+1,c) at r*W+c), or NULL
 *   lambda    uniform weight for whichever of d_wh / d_wv is NULL (>= 0)
 *   d_y0      optional H x W initial dual y^0 (a warm start), or NULL for y^0 = 0
 *   max_iters iteration limit (>= 0)
 *   gap_tol   per-pixel gap tolerance (> 0, or 0 to run exactly max_iters iterations)
 *   d_x       output H x W (must not overlap the inputs)
 *   iters_out, gap_out  optional HOST pointers: iterations run, final per-pixel gap
 * Returns TV_OK when converged, TV_ERR_NOT_CONVERGED (x still written) otherwise.
 */
tv_status tv2d_denoise(const float *d_img, int64_t H, int64_t W, const float *d_wh,
                       const float *d_wv, float lambda, const float *d_y0, int max_iters,
                       double gap_tol, float *d_x, int *iters_out, double *gap_out,
                       void *d_workspace, size_t workspace_bytes, tv_stream_t stream);

/* ------------------------------------------------------------ 2D, batched ---- */

/* One image of a batch (all pointers on the device; the caller owns them). */
typedef struct {
    const float *img;   /* H x W row-major noisy image */
    int64_t H, W;
    const float *wh;    /* H x (W-1) horizontal edge weights, or NULL */
    const float *wv;    /* (H-1) x W vertical edge weights, or NULL */
    float lambda;       /* uniform weight for whichever of wh / wv is NULL */
    const float *y0;    /* optional H x W initial dual (warm start), or NULL */
    float *x;           /* H x W output; must not alias the inputs */
    float *y_out;       /* optional H x W output: the final dual y (e.g. as a training target) */
} tv_image_desc;

/* Bytes of workspace tv2d_denoise_batched needs for these images (0 if malformed). */
size_t tv2d_batched_workspace_size(const tv_image_desc *imgs, int n_imgs, int max_iters);

/*
 * Denoise a batch of images of any sizes with the method of tv2d_denoise (Sec. 6.1,
 * eq. pd): every image iterates until its own per-pixel gap reaches gap_tol (or
 * max_iters). Each phase of an iteration is one launch over the chains of all
 * still-running images (the images' independent 1D subproblems, solved in
 * parallel); the iterations run inside one CUDA graph with a device-side loop
 * condition. `imgs` is a HOST array of n_imgs descriptors; iters_out and gap_out
 * are optional HOST arrays of n_imgs entries. Returns after the solve, TV_OK if
 * every image converged, TV_ERR_NOT_CONVERGED (outputs still written) otherwise.
 */
tv_status tv2d_denoise_batched(const tv_image_desc *imgs, int n_imgs, int max_iters,
                               double gap_tol, int *iters_out, double *gap_out,
                               void *d_workspace, size_t workspace_bytes, tv_stream_t stream);

/*
 * ROF denoising by the symmetric Lagrangian split of Sec. 6 (the form the paper uses
 * for stereo, here on the convex ROF model): x_h (rows) and x_v (columns) each carry half
 * of the data term and are coupled by a multiplier y,
 *     min_{x_h, x_v} max_y TV_h(x_h) + 1/4||x_h - f||^2 + TV_v(x_v) + 1/4||x_v - f||^2 + <x_h - x_v, y>,
 * with the primal-dual iteration of Sec. 6: tau_k = tau0 / k, sigma_k = 1 / (2 tau_k),
 * over-relaxation 1; start x_h = x_v = f, y = 0. Every check_every iterations (and at
 * max_iters) the per-pixel gap (P(xbar) - D(y)) / (H W) is evaluated, xbar = (x_h + x_v)/2,
 * D the Lagrangian dual (one extra row and column chain batch); the solve stops when it
 * is <= gap_tol (0: never early). d_x receives xbar. Arguments otherwise as
 * tv2d_denoise; workspace of tv2d_lagrangian_workspace_size bytes. Returns TV_OK or
 * TV_ERR_NOT_CONVERGED (x still written); synchronous at every gap check.
 */
size_t tv2d_lagrangian_workspace_size(int64_t H, int64_t W);
tv_status tv2d_denoise_lagrangian(const float *d_img, int64_t H, int64_t W, const float *d_wh,
                                  const float *d_wv, float lambda, float tau0, int max_iters,
                                  double gap_tol, int check_every, float *d_x, int *iters_out,
                                  double *gap_out, void *d_workspace, size_t workspace_bytes,
                                  tv_stream_t stream);

/*
 * 2D TV-l1 denoising (Sec. 6):  x* = argmin_x TV_h(x) + TV_v(x) + sum_p |x_p - f_p|,
 * weights as tv2d_denoise. Solved as the saddle point min_x max_y <x, y> + TV_h(x) +
 * ||x - f||_1 - TV_v^*(y) by the primal-dual iteration of eq. pd at constant steps
 * tau, sigma = 1/tau, theta = 1 (the model is not strongly convex), from x^0 = f, y^0 = 0:
 *   dual step    column chains (eq. prox-tv-conj) on c = y / sigma + xbar;
 *   primal step  row chains with piecewise-quadratic unaries (tv_chain_solve_pq) on
 *                xi = x - tau y, scaled by tau (a = 1, b = xi, alpha = tau, w = tau w_h);
 *   xbar = 2 x^{k+1} - x^k.
 * After every check_every-th iteration (and the last) the energy E = TV(x) + ||x - f||_1
 * is summed on the device (FP64, fixed order) and read back; the solve stops when two
 * consecutive checks differ by at most tol * E (tol = 0: run max_iters). tau in (0, inf);
 * 0.1 suits images with values in [0, 1] and lambda near 0.5. d_x receives x^k;
 * *iters_out the iterations run; *energy_out the last energy (either may be NULL).
 * Workspace of
 * tv2d_l1_workspace_size bytes. Returns TV_OK, or TV_ERR_NOT_CONVERGED when tol > 0 and
 * max_iters ran out (x still written); synchronous at every check.
 */
size_t tv2d_l1_workspace_size(int64_t H, int64_t W);
tv_status tv2d_denoise_l1(const float *d_img, int64_t H, int64_t W, const float *d_wh,
                          const float *d_wv, float lambda, float tau, int max_iters, double tol,
                          int check_every, float *d_x, int *iters_out, double *energy_out,
                          void *d_workspace, size_t workspace_bytes, tv_stream_t stream);

/* How the calling thread's last tv2d_denoise_batched ran its iterations: 1 as one
 * CUDA graph with a device-side loop condition, 0 replayed from the host (conditional
 * graph nodes unavailable, or disabled), -1 no batched solve yet. */
int tv2d_batched_last_mode(void);

/* Allow (1, the default) or forbid (0) the conditional-graph outer loop of
 * tv2d_denoise_batched, for every thread; forbidden, the same kernels are replayed
 * from the host (for tools that cannot follow a device-side loop, such as kernel
 * profilers). The environment variable TV_BATCHED_GRAPH=0 sets the initial value.
 * The two modes give bitwise identical results. */
tv_status tv_set_batched_graph(int on);

/*
 * Tuning knobs set by the autotuner (the paper has no counterpart): warps per block
 * of the batched phase kernels (1, 2, 4 or 8), and the largest chain batch solved
 * with one warp per chain instead of one thread per chain. 0 restores the defaults:
 * 4096 chains, and 2048 for tv_chain_solve batches of uniform rows of at least 64
 * nodes, a multiple of 4, with 16-byte aligned arrays (the one-thread-per-half kernel
 * stages those 16 bytes at a time and is the faster one from about 2048 chains on).
 * A value set here applies to every batch.
 */
tv_status tv_set_batched_warps(int warps_per_block);
tv_status tv_set_coop_max_chains(int64_t max_chains);
/* How a chain of 64 nodes or more is solved when its batch runs one warp per chain:
 * 0 by the whole warp from one end; 1 (the default) rooted at its middle node, the two
 * halves' forward passes run at once by the warp's two 16-lane halves (Algorithm 2
 * allows any root); 2 rooted at its middle node by two warps. All give the same
 * solution up to FP32 rounding. */
tv_status tv_set_coop_split(int mode);
/* How batches that run one thread per chain (tv_chain_solve with chains of 64 nodes or
 * more, and the thread path of tv2d_denoise_batched) solve a chain: 1 (the default)
 * rooted at the middle node, each half by its own thread (messages of up to 16
 * breakpoints on chip) and the root solved from both halves' messages (Algorithm 2
 * allows any root); 0 by one thread from one end (messages of up to 32 breakpoints on
 * chip). Longer messages are finished from the workspace either way. Both give the same
 * solution up to FP32 rounding. Read when a batched solve is planned. */
tv_status tv_set_thread_split(int on);
/* Whether tv2d_denoise, tv2d_denoise_lagrangian and tv2d_denoise_l1 launch the kernels
 * of their iterations, and the network's tensor-core convolutions and dual head
 * (tv_net_conv3x3 on tensor path 2, tv_net_conv3x3_grouped, tv_net_first_layer with
 * grouped output, tv_net_conv3x3_dual_head), with a programmatic dependency on the
 * previous kernel of the stream: 1 (the default) lets each kernel
 * become resident while its predecessor finishes, and the kernel waits in hardware for
 * that predecessor's completion and memory before it reads anything; 0 launches them
 * in plain stream order. The results are identical either way; only the gaps between
 * kernels differ. Read at each call. */
tv_status tv_set_programmatic_launch(int on);

/* ------------------------------------------ learned dual warm start (net) ---- */
/*
 * Building blocks of a small convolutional network that predicts a warm start y^0
 * for tv2d_denoise from the noisy image and lambda (the paper has no network: any
 * y^0 is a valid start of eq. pd). Tensors are NHWC bfloat16 (stored as uint16
 * bits) with 16 or 32 channels, zero-padded; weights are [cout][3][3][cin] bfloat16;
 * biases, pre-activations and gradients FP32. Convolutions are 3x3, stride 1, zero
 * padding 1 (cross-correlation), computed on BF16 tensor cores with FP32 accumulate.
 */
/* Which tensor-core path the forward convolutions take: 0 (the default) mma.sync
 * m16n8k16 (persistent blocks, 8 x 16 pixel tiles); 1 tcgen05.mma with TMEM accumulators
 * (128-pixel row tiles, two accumulators so that a tile's MMAs overlap the previous
 * tile's epilogue, one issuing thread per block). Both accumulate the same BF16 products
 * in FP32, in a different order. With 16 or 32 output channels each tcgen05 MMA is only
 * 128 x 32 x 16 and the forward pass of the network is faster on mma.sync (0.38 against
 * 0.53 ms at 1024 x 1024). The backward kernels always use mma.sync. */
tv_status tv_net_set_tensor_path(int mode);
/* Mode 2: the same tcgen05 GEMM per 128-pixel row tile, fed by TMA and run by warp roles
 * over vertical strips: a block walks runs of consecutive rows of one 128-pixel column, so
 * that each input row is loaded once per run (into a ring of six row slots) instead of
 * once per output row that reads it; one warp loads, one issues the MMAs into one of four
 * TMEM accumulators, four read the accumulators back, add the bias, apply the ReLU and
 * store. Measured at 1024 x 1024: 32 -> 32 channels 47 us against 66 us on mma.sync.
 * Every mbarrier wait of modes 1 and 2 gives up after a bounded number of polls (the tile
 * is then not written); tv_net_tensor_timeouts() returns how many waits gave up since the
 * library was loaded (-1 if the count cannot be read). */
int64_t tv_net_tensor_timeouts(void);

/* Inference layout ("grouped"): a C-channel BF16 activation stored as
 * [image][row][C/8 channel groups][pixel][8 channels], so that one group of one image row
 * is a contiguous run of W x 16 bytes (NHWC keeps a pixel's C channels together instead).
 * tv_net_conv3x3_grouped is tv_net_conv3x3 on this layout: x and act_out are grouped,
 * pre_out (FP32, may be NULL) stays NHWC. It always runs the tcgen05 kernel of mode 2 (a
 * row's TMA boxes are then 2048- and 32-byte runs instead of 130 16-byte pieces), whatever
 * the mode set by tv_net_set_tensor_path, and counts its timed-out waits in
 * tv_net_tensor_timeouts(). The same argument rules and errors as tv_net_conv3x3 apply. */
tv_status tv_net_conv3x3_grouped(const void *d_x, int B, int H, int W, int cin, const void *d_w,
                                 const float *d_bias, int cout, int relu, float *d_pre_out,
                                 void *d_act_out, tv_stream_t stream);

/* y = conv(x) + bias (bias may be NULL), optionally ReLU'd into act_out (BF16, may be
 * NULL); pre_out (FP32, may be NULL) receives the value before the ReLU; at least one of
 * the two outputs is given. All tensor pointers 16-byte aligned; B <= 65535. */
tv_status tv_net_conv3x3(const void *d_x, int B, int H, int W, int cin, const void *d_w,
                         const float *d_bias, int cout, int relu, float *d_pre_out,
                         void *d_act_out, tv_stream_t stream);
/* dx = (conv^T dy) * (mask_pre > 0): gradient with respect to the input of a
 * convolution whose input was ReLU(mask_pre). scratch_w: cout*9*cin BF16 entries. */
tv_status tv_net_conv3x3_backward_data(const void *d_dy, int B, int H, int W, int cout,
                                       const void *d_w, int cin, const float *d_mask_pre,
                                       void *d_dx, void *d_scratch_w, tv_stream_t stream);
/* Bytes of the workspace that tv_net_conv3x3_backward_weight and tv_net_dual_head
 * (with a loss) need for a B x H x W batch on the current device (0 for a bad shape). */
size_t tv_net_workspace_size(int B, int H, int W);
/* dw += sum_p dy[p] x[p+tap]^T and db += sum_p dy[p] (FP32, accumulated: zero them first;
 * d_db may be NULL). Per-block partial sums go to the workspace and are added in a fixed
 * order, so the result is deterministic. */
tv_status tv_net_conv3x3_backward_weight(const void *d_x, const void *d_dy, int B, int H, int W,
                                         int cin, int cout, float *d_dw, float *d_db,
                                         void *d_ws, size_t ws_bytes, tv_stream_t stream);
/* Network input: channel 0 the image f, channel 1 its lambda (per image), 2..15 zero. */
tv_status tv_net_pack_input(const float *d_f, int B, int H, int W, const float *d_lam, void *d_x,
                            tv_stream_t stream);
/* Output head: p_v = lambda * tanh(o) on vertical edges (o = channel 0 of a 16-channel
 * FP32 tensor), y = D_v^T p_v (y[r] = p[r-1] - p[r]), a dual-feasible warm start. With
 * d_target: *d_loss = mean (y - target)^2 if d_loss (block partials in the workspace,
 * summed in a fixed order) and, if d_grad_o, its gradient with respect to o (BF16, 16
 * channels, channels 1..15 zero). d_ws may be NULL when d_loss is. */
/* Inference-only form of the first layer, on the CUDA cores. The network's input has two
 * non-zero channels (the image and its lambda, 2..15 zero), so the first layer needs no
 * packed input: tv_net_first_layer reads the FP32 images d_f (B x H x W) and d_lam, rounds
 * both to BF16 as tv_net_pack_input would, and writes the ReLU'd 32-channel BF16
 * activation (16-byte aligned) of the 16 -> 32 layer with weights d_w ([32][3][3][16]
 * BF16; input channels 2..15 are not read) and bias d_bias (may be NULL). It equals
 * tv_net_pack_input followed by tv_net_conv3x3 up to the order of FP32 sums. With
 * grouped != 0 the activation is written in the grouped layout (above) instead of NHWC,
 * and the layer runs on tcgen05 (the kernel of tv_net_conv3x3_grouped, whose loading warp
 * builds each BF16 input row from f and lambda in shared memory); with grouped == 0 on the
 * CUDA cores. */
tv_status tv_net_first_layer(const float *d_f, int B, int H, int W, const float *d_lam,
                             const void *d_w, const float *d_bias, void *d_act_out, int grouped,
                             tv_stream_t stream);
/* The network's last layer fused with its head, for inference: the cin -> 16 convolution
 * of the grouped activation d_x (weights d_w [16][3][3][cin] BF16, bias d_bias, may be
 * NULL) whose epilogue keeps only channel 0, o, and writes d_p = lambda tanh(o) on the
 * vertical edges (rows 0 .. H-2; 0 on each image's last row; B x H x W FP32), followed by
 * d_y = D_v^T p (y[r] = p[r-1] - p[r]), which equals tv_net_dual_head on that o. cin is 16
 * or 32; x and w 16-byte aligned; timed-out waits count in tv_net_tensor_timeouts(). */
tv_status tv_net_conv3x3_dual_head(const void *d_x, int B, int H, int W, int cin, const void *d_w,
                                   const float *d_bias, const float *d_lam, float *d_p, float *d_y,
                                   tv_stream_t stream);
tv_status tv_net_dual_head(const float *d_o, int B, int H, int W, const float *d_lam,
                           const float *d_target, float *d_y, float *d_loss, void *d_grad_o,
                           void *d_ws, size_t ws_bytes, tv_stream_t stream);
/* out[i] = bfloat16(a[i]) (round to nearest even), i < n. */
tv_status tv_net_cast_bf16(const float *d_a, int64_t n, void *d_out, tv_stream_t stream);
/* One Adam step on n FP32 parameters (step counts from 1); the gradient is read and
 * then cleared; w_bf16 (may be NULL) receives a BF16 copy of the new weights. */
tv_status tv_net_adam(float *d_w, float *d_m, float *d_v, float *d_g, int64_t n, float lr,
                      float beta1, float beta2, float eps, int step, void *d_w_bf16,
                      tv_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif
