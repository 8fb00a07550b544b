/*
 * Plain FP64 CPU oracle for total variation on chains and for 2D TV-l2 (ROF)
 * denoising by Lagrangian decomposition.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct reference
 * that the CUDA path is checked against. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, headers, tables or
 * constants with the CUDA library.
 *
 * Problem (eq. 1D-ROF, Sec. 6.1; Sec. 4.1 with a_i = 1, b_i = c_i):
 *     x* = argmin_x  sum_i 1/2 (x_i - c_i)^2 + sum_{i<n} w_i |x_{i+1} - x_i|
 * Edge i joins nodes i and i+1 (0-based here); w has one entry per edge.
 *
 * Algorithm: Algorithm 2 (convex DP with subgradient messages), specialised as
 * in Sec. 4.1: messages are piecewise-linear, stored as a sequence of
 * breakpoints lambda_p with an implicit slope s_p (true slope s_p + abar_i,
 * abar_i = sum_{k<=i} a_k = i for a_k = 1) in a two-ended array started in its
 * middle; the forward pass records lambda^-_i and lambda^+_i, the backward pass
 * clips x_i = clip(x_{i+1}, lambda^-_i, lambda^+_i).
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *  - After the left scan the segment to the right of the new breakpoint
 *    lambda^- lies inside old segment ell, so it keeps slope s_ell (the printed
 *    "s_{ell+1}" is read as an off-by-one).
 *  - In the right-scan recursion the printed "alpha_t" is read as lambda_t.
 *  - Node 1 has no incoming message: lambda^-_1 = c_1 - w_1, lambda^+_1 = c_1 + w_1.
 *  - The virtual root edge has w = 0 (Algorithm 2, first step); x_n is the
 *    midpoint of the (degenerate) interval [lambda^-_n, lambda^+_n].
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TVO_OK 0
#define TVO_ERR_INVALID 1
#define TVO_ERR_NOMEM 5
#define TVO_NOT_CONVERGED 3

/* One breakpoint of the current message: X-coordinate lambda_p and the stored
 * slope s_p of the segment to its right (Sec. 4.1, "2 floating points per
 * breakpoint"). */
typedef struct {
    double lam;
    double s;
} tvo_bp;

static double edge_w(const double *w, double lam, int64_t i) { return w ? w[i] : lam; }

/*
 * Forward and backward pass on one chain of length n.
 * c: n unary targets; w: n-1 edge weights or NULL (then every edge has weight lam).
 * x: n outputs. lo, hi: optional n-entry records of lambda^-_i, lambda^+_i.
 * D: scratch of at least 2n+2 breakpoints. Returns the largest sequence length seen.
 */
static int64_t chain_solve_core(int64_t n, const double *c, const double *w, double lam,
                                double *x, double *lo, double *hi, tvo_bp *D)
{
    if (n <= 0) return 0;
    if (n == 1) {
        x[0] = c[0];
        if (lo) lo[0] = c[0];
        if (hi) hi[0] = c[0];
        return 0;
    }
    /* The record of lambda^- lives in x (Sec. 4.1, last paragraph); lambda^+ in hi_rec. */
    double *lam_minus = x;
    double *lam_plus = hi ? hi : (double *)malloc(sizeof(double) * (size_t)n);
    if (!lam_plus) return -1;

    /* Node 1 (index 0): m^_1(z) = z - c_1 has slope a_1 = 1 everywhere. */
    double w0 = edge_w(w, lam, 0);
    int64_t front = n, back = n + 1; /* the sequence occupies D[front..back] */
    D[front].lam = c[0] - w0;
    D[front].s = 0.0;           /* true slope 1 = s + abar_1 between the two breakpoints */
    D[back].lam = c[0] + w0;
    D[back].s = -1.0;           /* right end: -abar_1, true slope 0 in m_{12} */
    lam_minus[0] = D[front].lam;
    lam_plus[0] = D[back].lam;
    int64_t max_len = 2;
    double w_prev = w0;

    for (int64_t i = 1; i < n; ++i) {
        const double abar = (double)(i + 1);                 /* abar_i = abar_{i-1} + a_i */
        const double wi = (i < n - 1) ? edge_w(w, lam, i) : 0.0; /* root edge: w = 0 */
        const double ci = c[i];

        /* Left scan: largest ell with m^_i(lambda_ell) < -w_i. Values of m^_i at the
         * breakpoints follow the forward recursion from the first one, whose incoming
         * message value is -w_{i-1}. */
        int64_t p = front;
        double v = -w_prev + D[p].lam - ci;
        int64_t last_popped;       /* entries D[front..last_popped] are removed */
        double lm, lm_s;
        if (v >= -wi) {
            /* ell = 0: lambda^- lies on the left end segment, true slope a_i = 1. */
            last_popped = front - 1;
            lm = D[p].lam - (v + wi);
            lm_s = 1.0 - abar;
        } else {
            while (p < back) {
                double vq = v + (D[p].s + abar) * (D[p + 1].lam - D[p].lam);
                if (vq < -wi) {
                    ++p;
                    v = vq;
                } else {
                    break;
                }
            }
            /* m^_i(lambda_ell) = v < -w_i; lambda^- lies in segment ell, slope s_ell + abar. */
            last_popped = p;
            lm = D[p].lam + (-wi - v) / (D[p].s + abar);
            lm_s = D[p].s;
        }

        /* Right scan over the original breakpoints with index > ell: smallest r with
         * m^_i(lambda_r) > w_i, using the backward recursion from the last breakpoint,
         * whose incoming message value is +w_{i-1}. */
        double hp;
        int64_t new_back_last; /* last original entry that is kept */
        if (back > last_popped) {
            int64_t q = back;
            double vr = w_prev + D[q].lam - ci;
            if (vr <= wi) {
                /* r = t+1: lambda^+ lies on the right end segment, true slope 1. */
                hp = D[q].lam + (wi - vr);
                new_back_last = back;
            } else {
                for (;;) {
                    if (q - 1 > last_popped) {
                        double slope = D[q - 1].s + abar;
                        double vprev = vr - slope * (D[q].lam - D[q - 1].lam);
                        if (vprev > wi) {
                            --q;
                            vr = vprev;
                            continue;
                        }
                        hp = D[q].lam - (vr - wi) / slope;
                    } else {
                        /* The segment to the left of lambda_r starts at the new lambda^-. */
                        hp = D[q].lam - (vr - wi) / (lm_s + abar);
                    }
                    break;
                }
                new_back_last = q - 1;
            }
        } else {
            /* Every original breakpoint lies left of lambda^-: m^_i is linear to its right. */
            hp = lm + (wi + wi) / (lm_s + abar);
            new_back_last = last_popped;
        }

        /* New sequence (-abar_i, lambda^-, s_ell, lambda_{ell+1}, ..., s_{r-1}, lambda^+, -abar_i). */
        front = last_popped;
        D[front].lam = lm;
        D[front].s = lm_s;
        back = (new_back_last > front ? new_back_last : front) + 1;
        D[back].lam = hp;
        D[back].s = -abar;
        if (back - front + 1 > max_len) max_len = back - front + 1;

        lam_minus[i] = lm;
        lam_plus[i] = hp;
        w_prev = wi;
    }

    if (lo) memcpy(lo, lam_minus, sizeof(double) * (size_t)n);
    /* Backward pass (Algorithm 2, last loop): root value, then clip toward the leaves. */
    x[n - 1] = 0.5 * (lam_minus[n - 1] + lam_plus[n - 1]);
    for (int64_t i = n - 2; i >= 0; --i) {
        double v = x[i + 1];
        if (v < lam_minus[i]) v = lam_minus[i];
        if (v > lam_plus[i]) v = lam_plus[i];
        x[i] = v;
    }
    if (!hi) free(lam_plus);
    return max_len;
}

/* Single chain, optional lambda^+- records (lo, hi may be NULL) and the largest
 * message length. Returns TVO_OK or an error code. */
int tvo_chain_solve(int64_t n, const double *c, const double *w, double lam, double *x,
                    double *lo, double *hi, int64_t *max_len)
{
    if (n < 0 || !c || !x) return TVO_ERR_INVALID;
    tvo_bp *D = (tvo_bp *)malloc(sizeof(tvo_bp) * (size_t)(2 * n + 2));
    if (!D) return TVO_ERR_NOMEM;
    int64_t m = chain_solve_core(n, c, w, lam, x, lo, hi, D);
    free(D);
    if (m < 0) return TVO_ERR_NOMEM;
    if (max_len) *max_len = m;
    return TVO_OK;
}

/* ---------------- the general convex chain (Sec. 4, Sec. 4.1) ----------------
 *
 * Unaries f_i(x) = a_i x^2 / 2 - b_i x with a_i > 0 (Sec. 4.1), pairwise terms on
 * d = x_{i+1} - x_i: f_i(d) = w^-_i d for d < 0 and w^+_i d for d >= 0, with
 * w^-_i <= w^+_i (Sec. 4). Algorithm 2: m^_i(z) = m_{i-1,i}(z) + a_i z - b_i
 * (transformation (a)), m_{i,i+1} = clip_[w^-_i, w^+_i](m^_i) (transformation (b)),
 * lambda^-_i and lambda^+_i where m^_i reaches w^-_i and w^+_i; the root edge has
 * w^- = w^+ = 0. The stored slope s_p has true slope s_p + abar_i with
 * abar_i = sum_{k<=i} a_k (Sec. 4.1). TV-l2 is a_i = 1, b_i = c_i, w^-_i = -w_i,
 * w^+_i = w_i.
 */
static int64_t chain_general_core(int64_t n, const double *a, const double *b, const double *wlo,
                                  const double *whi, double *x, double *lo, double *hi, tvo_bp *D)
{
    if (n <= 0) return 0;
    if (n == 1) {
        x[0] = b[0] / a[0];
        if (lo) lo[0] = x[0];
        if (hi) hi[0] = x[0];
        return 0;
    }
    double *lam_minus = (double *)malloc(sizeof(double) * (size_t)n);
    double *lam_plus = (double *)malloc(sizeof(double) * (size_t)n);
    if (!lam_minus || !lam_plus) {
        free(lam_minus);
        free(lam_plus);
        return -1;
    }
    /* Node 0: m^_0(z) = a_0 z - b_0. */
    double abar = a[0];
    int64_t front = n, back = n + 1;
    D[front].lam = (b[0] + wlo[0]) / a[0];
    D[front].s = a[0] - abar; /* true slope a_0 between the two breakpoints */
    D[back].lam = (b[0] + whi[0]) / a[0];
    D[back].s = -abar;        /* true slope 0: the clipped flat right end */
    lam_minus[0] = D[front].lam;
    lam_plus[0] = D[back].lam;
    int64_t max_len = 2;
    double wl_prev = wlo[0], wh_prev = whi[0];

    for (int64_t i = 1; i < n; ++i) {
        const double ai = a[i], bi = b[i];
        abar += ai;
        const double wl = (i < n - 1) ? wlo[i] : 0.0; /* root edge */
        const double wh = (i < n - 1) ? whi[i] : 0.0;

        /* Left scan: forward recursion from the first breakpoint, where the incoming
         * message has its left value w^-_{i-1}. */
        int64_t p = front;
        double v = wl_prev + ai * D[p].lam - bi;
        int64_t last_popped;
        double lm, lm_s;
        if (v >= wl) {
            /* lambda^- on the left end segment, true slope a_i */
            last_popped = front - 1;
            lm = D[p].lam + (wl - v) / ai;
            lm_s = ai - abar;
        } else {
            while (p < back) {
                double vq = v + (D[p].s + abar) * (D[p + 1].lam - D[p].lam);
                if (vq < wl) {
                    ++p;
                    v = vq;
                } else {
                    break;
                }
            }
            last_popped = p;
            lm = D[p].lam + (wl - v) / (D[p].s + abar);
            lm_s = D[p].s;
        }

        /* Right scan over the breakpoints kept by the left scan: backward recursion
         * from the last breakpoint, where the incoming message has its right value
         * w^+_{i-1}. */
        double hp;
        int64_t new_back_last;
        if (back > last_popped) {
            int64_t q = back;
            double vr = wh_prev + ai * D[q].lam - bi;
            if (vr <= wh) {
                /* lambda^+ on the right end segment, true slope a_i */
                hp = D[q].lam + (wh - vr) / ai;
                new_back_last = back;
            } else {
                for (;;) {
                    if (q - 1 > last_popped) {
                        double slope = D[q - 1].s + abar;
                        double vprev = vr - slope * (D[q].lam - D[q - 1].lam);
                        if (vprev > wh) {
                            --q;
                            vr = vprev;
                            continue;
                        }
                        hp = D[q].lam - (vr - wh) / slope;
                    } else {
                        hp = D[q].lam - (vr - wh) / (lm_s + abar);
                    }
                    break;
                }
                new_back_last = q - 1;
            }
        } else {
            hp = lm + (wh - wl) / (lm_s + abar);
            new_back_last = last_popped;
        }

        front = last_popped;
        D[front].lam = lm;
        D[front].s = lm_s;
        back = (new_back_last > front ? new_back_last : front) + 1;
        D[back].lam = hp;
        D[back].s = -abar;
        if (back - front + 1 > max_len) max_len = back - front + 1;
        lam_minus[i] = lm;
        lam_plus[i] = hp;
        wl_prev = wl;
        wh_prev = wh;
    }

    x[n - 1] = 0.5 * (lam_minus[n - 1] + lam_plus[n - 1]);
    for (int64_t i = n - 2; i >= 0; --i) {
        double v = x[i + 1];
        if (v < lam_minus[i]) v = lam_minus[i];
        if (v > lam_plus[i]) v = lam_plus[i];
        x[i] = v;
    }
    if (lo) memcpy(lo, lam_minus, sizeof(double) * (size_t)n);
    if (hi) memcpy(hi, lam_plus, sizeof(double) * (size_t)n);
    free(lam_minus);
    free(lam_plus);
    return max_len;
}

/* General chains in a CSR batch (one thread; a, b, wlo, whi laid out like x, the
 * entries at a chain's last node of wlo/whi unused). */
int tvo_chain_solve_general_batch(const double *a, const double *b, const double *wlo,
                                  const double *whi, const int64_t *offsets, int64_t num_chains,
                                  double *x)
{
    if (num_chains < 0 || !offsets) return TVO_ERR_INVALID;
    int64_t nmax = 0;
    for (int64_t k = 0; k < num_chains; ++k) {
        const int64_t len = offsets[k + 1] - offsets[k];
        if (len < 0) return TVO_ERR_INVALID;
        if (len > nmax) nmax = len;
    }
    tvo_bp *D = (tvo_bp *)malloc(sizeof(tvo_bp) * (size_t)(2 * nmax + 4));
    if (!D) return TVO_ERR_NOMEM;
    for (int64_t k = 0; k < num_chains; ++k) {
        const int64_t o = offsets[k], len = offsets[k + 1] - offsets[k];
        for (int64_t i = 0; i < len; ++i)
            if (!(a[o + i] > 0.0) || (i < len - 1 && !(wlo[o + i] <= whi[o + i]))) {
                free(D);
                return TVO_ERR_INVALID;
            }
        if (chain_general_core(len, a + o, b + o, wlo + o, whi + o, x + o, NULL, NULL, D) < 0) {
            free(D);
            return TVO_ERR_NOMEM;
        }
    }
    free(D);
    return TVO_OK;
}

/* ---------------- batches of contiguous chains (CSR offsets), threaded ---------------- */

typedef struct {
    const double *c, *w;
    double lam;
    const int64_t *offsets;
    int64_t begin, end;
    double *x;
    int64_t max_len;
    int status;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *j = (batch_job *)arg;
    int64_t maxn = 0;
    for (int64_t k = j->begin; k < j->end; ++k) {
        int64_t n = j->offsets[k + 1] - j->offsets[k];
        if (n > maxn) maxn = n;
    }
    tvo_bp *D = (tvo_bp *)malloc(sizeof(tvo_bp) * (size_t)(2 * maxn + 2));
    if (!D) {
        j->status = TVO_ERR_NOMEM;
        return NULL;
    }
    j->max_len = 0;
    for (int64_t k = j->begin; k < j->end; ++k) {
        int64_t o = j->offsets[k], n = j->offsets[k + 1] - o;
        /* w is indexed per node like c; the entry at a chain's last node is unused. */
        int64_t m = chain_solve_core(n, j->c + o, j->w ? j->w + o : NULL, j->lam, j->x + o, NULL,
                                     NULL, D);
        if (m < 0) {
            j->status = TVO_ERR_NOMEM;
            break;
        }
        if (m > j->max_len) j->max_len = m;
    }
    free(D);
    return NULL;
}

int tvo_chain_solve_batch(const double *c, const double *w, double lam, const int64_t *offsets,
                          int64_t num_chains, double *x, int nthreads, int64_t *max_len)
{
    if (num_chains < 0 || !offsets) return TVO_ERR_INVALID;
    for (int64_t k = 0; k < num_chains; ++k)
        if (offsets[k + 1] < offsets[k]) return TVO_ERR_INVALID;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > num_chains) nthreads = num_chains > 0 ? (int)num_chains : 1;
    batch_job *jobs = (batch_job *)calloc((size_t)nthreads, sizeof(batch_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs);
        free(th);
        return TVO_ERR_NOMEM;
    }
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (batch_job){c, w, lam, offsets, num_chains * t / nthreads,
                              num_chains * (t + 1) / nthreads, x, 0, TVO_OK};
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
    batch_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    int st = TVO_OK;
    int64_t m = 0;
    for (int t = 0; t < nthreads; ++t) {
        if (jobs[t].status != TVO_OK) st = jobs[t].status;
        if (jobs[t].max_len > m) m = jobs[t].max_len;
    }
    if (max_len) *max_len = m;
    free(jobs);
    free(th);
    return st;
}

/* ---------------- vector-Jacobian product of the chain prox ---------------- */

/*
 * Gradient of L(x*(c, w)) given g = dL/dx*, on one chain.
 * Away from degenerate points the optimality conditions of eq. 1D-ROF give, on
 * every maximal run S = [l..r] of equal values ("segment"),
 *     x_S = mean(c_S) + (u_r - u_{l-1}) / |S|,   u_e = w_e * sign(x_{e+1} - x_e)
 * at the jump edges bounding S (u = 0 past the chain ends). Hence
 *     dL/dc_j = mean_{i in S(j)} g_i,
 *     dL/dw_e = sign_e * (mean_{S left of e} g - mean_{S right of e} g) at a jump
 *               edge e, and 0 on edges inside a segment.
 * Two neighbours belong to one segment when |x_{e+1} - x_e| <= fuse_tol.
 * grad_w (n-1 entries) may be NULL.
 */
int tvo_chain_vjp(int64_t n, const double *x, const double *g, double fuse_tol, double *grad_c,
                  double *grad_w)
{
    if (n < 0 || (n > 0 && (!x || !g || !grad_c))) return TVO_ERR_INVALID;
    int64_t l = 0;
    double prev_mean = 0.0;
    int64_t prev_edge = -1; /* jump edge that closes the previous segment */
    while (l < n) {
        int64_t r = l;
        while (r + 1 < n && fabs(x[r + 1] - x[r]) <= fuse_tol) ++r;
        double sum = 0.0;
        for (int64_t i = l; i <= r; ++i) sum += g[i];
        double mean = sum / (double)(r - l + 1);
        for (int64_t i = l; i <= r; ++i) grad_c[i] = mean;
        if (grad_w) {
            for (int64_t e = l; e < r; ++e) grad_w[e] = 0.0;
            if (prev_edge >= 0) {
                double sgn = x[prev_edge + 1] > x[prev_edge] ? 1.0 : -1.0;
                grad_w[prev_edge] = sgn * (prev_mean - mean);
            }
        }
        prev_mean = mean;
        prev_edge = r;
        l = r + 1;
    }
    return TVO_OK;
}

/* ---------------- 2D TV-l2 by Lagrangian decomposition (eq. pd) ---------------- */

typedef struct {
    int64_t count, len;     /* number of chains and their length */
    int64_t stride_chain;   /* distance between the first nodes of consecutive chains */
    int64_t stride_node;    /* distance between consecutive nodes of one chain */
    const double *c;        /* unary targets, image layout */
    const double *w;        /* edge weights: chain k edge e at w[k*w_chain + e*w_node] */
    int64_t w_chain, w_node;
    double w_scale;         /* every weight is multiplied by this */
    double lam;             /* used when w == NULL */
    double *x;              /* solution, image layout */
    int64_t begin, end;
    int status;
} phase_job;

static void *phase_worker(void *arg)
{
    phase_job *j = (phase_job *)arg;
    int64_t n = j->len;
    double *cb = (double *)malloc(sizeof(double) * (size_t)n);
    double *wb = (double *)malloc(sizeof(double) * (size_t)(n > 1 ? n - 1 : 1));
    double *xb = (double *)malloc(sizeof(double) * (size_t)n);
    tvo_bp *D = (tvo_bp *)malloc(sizeof(tvo_bp) * (size_t)(2 * n + 2));
    if (!cb || !wb || !xb || !D) {
        j->status = TVO_ERR_NOMEM;
    } else {
        for (int64_t k = j->begin; k < j->end; ++k) {
            for (int64_t i = 0; i < n; ++i) cb[i] = j->c[k * j->stride_chain + i * j->stride_node];
            for (int64_t e = 0; e + 1 < n; ++e)
                wb[e] = j->w_scale * (j->w ? j->w[k * j->w_chain + e * j->w_node] : j->lam);
            if (chain_solve_core(n, cb, wb, 0.0, xb, NULL, NULL, D) < 0) {
                j->status = TVO_ERR_NOMEM;
                break;
            }
            for (int64_t i = 0; i < n; ++i) j->x[k * j->stride_chain + i * j->stride_node] = xb[i];
        }
    }
    free(cb);
    free(wb);
    free(xb);
    free(D);
    return NULL;
}

/* Solve every chain of one phase (all rows or all columns) on nthreads threads. */
static int run_phase(phase_job proto, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > proto.count) nthreads = (int)proto.count;
    phase_job jobs[256];
    pthread_t th[256];
    if (nthreads > 256) nthreads = 256;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = proto;
        jobs[t].begin = proto.count * t / nthreads;
        jobs[t].end = proto.count * (t + 1) / nthreads;
        jobs[t].status = TVO_OK;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, phase_worker, &jobs[t]);
    phase_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < nthreads; ++t)
        if (jobs[t].status != TVO_OK) return jobs[t].status;
    return TVO_OK;
}

/* Row phase: x = argmin TV_h(x) + k/2 ||x - c||^2 solved as chains with c and
 * weights w_h / k (eq. 1D-ROF after dividing by k). */
static int row_prox(int H, int W, const double *c, const double *wh, double lam, double k,
                    double *x, int nthreads)
{
    phase_job p = {H, W, W, 1, c, wh, W - 1, 1, 1.0 / k, lam, x, 0, 0, TVO_OK};
    return run_phase(p, nthreads);
}

/* Column phase: the same along columns with weights w_v / k. */
static int col_prox(int H, int W, const double *c, const double *wv, double lam, double k,
                    double *x, int nthreads)
{
    phase_job p = {W, H, 1, W, c, wv, 1, W, 1.0 / k, lam, x, 0, 0, TVO_OK};
    return run_phase(p, nthreads);
}

/*
 * Primal objective P(x) = 1/2 ||x - f||^2 + TV_h(x) + TV_v(x) of the ROF model
 * (Sec. 6.1). wh: H*(W-1) (edge (r,c)-(r,c+1) at r*(W-1)+c); wv: (H-1)*W (edge
 * (r,c)-(r+1,c) at r*W+c); NULL means the uniform weight lam.
 */
double tvo_rof_primal(int H, int W, const double *f, const double *wh, const double *wv,
                      double lam, const double *x)
{
    double s = 0.0;
    for (int64_t i = 0; i < (int64_t)H * W; ++i) s += 0.5 * (x[i] - f[i]) * (x[i] - f[i]);
    for (int r = 0; r < H; ++r)
        for (int c = 0; c + 1 < W; ++c)
            s += (wh ? wh[(int64_t)r * (W - 1) + c] : lam) *
                 fabs(x[(int64_t)r * W + c + 1] - x[(int64_t)r * W + c]);
    for (int r = 0; r + 1 < H; ++r)
        for (int c = 0; c < W; ++c)
            s += (wv ? wv[(int64_t)r * W + c] : lam) *
                 fabs(x[(int64_t)(r + 1) * W + c] - x[(int64_t)r * W + c]);
    return s;
}

/*
 * Accelerated primal-dual iteration (eq. pd) on the saddle-point problem
 * eq. rof-saddle, with the two proximal maps of Sec. 6.1:
 *   eta     = y^k + sigma_k (x^k + theta_{k-1} (x^k - x^{k-1}))
 *   xhat    = argmin TV_v(x) + sigma_k/2 ||x - eta/sigma_k||^2   (column chains)
 *   y^{k+1} = eta - sigma_k xhat                                  (eq. prox-tv-conj)
 *   xi      = x^k - tau_k y^{k+1}
 *   x^{k+1} = argmin TV_h(x) + (1+1/tau_k)/2 ||x - (f + xi/tau_k)/(1+1/tau_k)||^2  (row chains)
 *   theta_k = 1/sqrt(1 + 2 gamma tau_k), tau_{k+1} = theta_k tau_k,
 *   sigma_{k+1} = sigma_k / theta_k, with gamma = 1 and tau_0 sigma_0 = 1.
 * Start: y^0 = y0 (or 0) and x^0 = x^{-1} = argmin TV_h(x) + 1/2 ||x - (f - y^0)||^2.
 * Gap after step k (a reading: the paper plots convergence but defines no gap):
 *   G_k = P(x^{k+1}) - D(p_h, p_v), with the dual-feasible edge fields that the two
 *   chain solves certify, for which f - D_h^T p_h - D_v^T p_v = x^{k+1} + (x^{k+1}-x^k)/tau_k:
 *   G_k = 1/2||x^{k+1}-f||^2 + TV(x^{k+1}) - 1/2||f||^2 + 1/2||x^{k+1} + (x^{k+1}-x^k)/tau_k||^2.
 * Stops at the first k with G_k / (H W) <= tol; returns x^{k+1} and k+1 iterations.
 * gap_trace (max_iters entries, optional) receives G_k / (H W).
 */
int tvo_tv2d_pd(int H, int W, const double *f, const double *wh, const double *wv, double lam,
                const double *y0, int max_iters, double tol, double tau0, int nthreads,
                double *x_out, int *iters_out, double *gap_trace, double *y_out)
{
    if (H < 1 || W < 1 || !f || !x_out || max_iters < 0 || !(tau0 > 0.0)) return TVO_ERR_INVALID;
    int64_t N = (int64_t)H * W;
    double *x = (double *)calloc((size_t)N, sizeof(double));
    double *xp = (double *)calloc((size_t)N, sizeof(double));
    double *y = (double *)calloc((size_t)N, sizeof(double));
    double *c = (double *)calloc((size_t)N, sizeof(double));
    double *xh = (double *)calloc((size_t)N, sizeof(double));
    int st = TVO_OK;
    if (!x || !xp || !y || !c || !xh) {
        st = TVO_ERR_NOMEM;
        goto done;
    }
    if (y0) memcpy(y, y0, sizeof(double) * (size_t)N);
    for (int64_t i = 0; i < N; ++i) c[i] = f[i] - y[i];
    if ((st = row_prox(H, W, c, wh, lam, 1.0, x, nthreads)) != TVO_OK) goto done;
    memcpy(xp, x, sizeof(double) * (size_t)N);

    double tau = tau0, sigma = 1.0 / tau0, theta_prev = 1.0;
    double half_f2 = 0.0;
    for (int64_t i = 0; i < N; ++i) half_f2 += 0.5 * f[i] * f[i];
    int k;
    st = TVO_NOT_CONVERGED;
    for (k = 0; k < max_iters; ++k) {
        /* dual step: column chains via the Moreau identity */
        for (int64_t i = 0; i < N; ++i) {
            double eta = y[i] + sigma * (x[i] + theta_prev * (x[i] - xp[i]));
            y[i] = eta; /* eta kept in y until the chain solve returns */
            c[i] = eta / sigma;
        }
        int s2 = col_prox(H, W, c, wv, lam, sigma, xh, nthreads);
        if (s2 != TVO_OK) {
            st = s2;
            goto done;
        }
        for (int64_t i = 0; i < N; ++i) y[i] = y[i] - sigma * xh[i];
        /* primal step: row chains */
        double kk = 1.0 + 1.0 / tau;
        for (int64_t i = 0; i < N; ++i) {
            double xi = x[i] - tau * y[i];
            c[i] = (f[i] + xi / tau) / kk;
        }
        memcpy(xp, x, sizeof(double) * (size_t)N);
        s2 = row_prox(H, W, c, wh, lam, kk, x, nthreads);
        if (s2 != TVO_OK) {
            st = s2;
            goto done;
        }
        /* gap of (x^{k+1}, certified duals) */
        double g = tvo_rof_primal(H, W, f, wh, wv, lam, x) - half_f2;
        for (int64_t i = 0; i < N; ++i) {
            double z = x[i] + (x[i] - xp[i]) / tau;
            g += 0.5 * z * z;
        }
        if (gap_trace) gap_trace[k] = g / (double)N;
        /* step sizes of the accelerated variant */
        double theta = 1.0 / sqrt(1.0 + 2.0 * tau);
        tau = theta * tau;
        sigma = sigma / theta;
        theta_prev = theta;
        if (g / (double)N <= tol) {
            st = TVO_OK;
            ++k;
            break;
        }
    }
    if (iters_out) *iters_out = k;
    memcpy(x_out, x, sizeof(double) * (size_t)N);
    if (y_out) memcpy(y_out, y, sizeof(double) * (size_t)N);
done:
    free(x);
    free(xp);
    free(y);
    free(c);
    free(xh);
    return st;
}


/* ---------------- the symmetric Lagrangian form (Sec. 6) on the ROF model ----------------
 *
 * min_{x_h, x_v} max_y Psi_h(x_h) + Psi_v(x_v) + <x_h - x_v, y>, with
 * Psi_{h,v}(x) = TV_{h,v}(x) + 1/4 ||x - f||^2 (each half carries half of the data term),
 * solved by the primal-dual iteration printed in Sec. 6 for this split:
 *   x_h^{k+1} = prox_{tau_k Psi_h}(x_h^k - tau_k ybar^k)        (row chains)
 *   x_v^{k+1} = prox_{tau_k Psi_v}(x_v^k + tau_k ybar^k)        (column chains)
 *   y^{k+1}   = y^k + sigma_k (x_h^{k+1} - x_v^{k+1})
 *   ybar^{k+1} = y^{k+1} + theta (y^{k+1} - y^k)
 * with tau_k = tau0 / k (k = 1, 2, ...), sigma_k = 1 / (tau_k L^2), L^2 = 2, theta = 1.
 * prox_{tau Psi_h}(z) = argmin TV_h(x) + 1/4 ||x - f||^2 + 1/(2 tau) ||x - z||^2 is a chain
 * problem with curvature a = 1/2 + 1/tau, target c = (f/2 + z/tau) / a and weights w / a.
 * Start: x_h = x_v = f, y = ybar = 0.
 * Gap (a reading: the paper gives none for this form): every check_every iterations and
 * at the last one, P(xbar) - D(y) with xbar = (x_h + x_v)/2, P the ROF energy and the
 * Lagrangian dual D(y) = min_x [TV_h(x) + 1/4||x - f||^2 + <x, y>]
 *                      + min_x [TV_v(x) + 1/4||x - f||^2 - <x, y>] <= min P;
 * each minimum is a chain problem with target f -+ 2y and weights 2w. Stops when the
 * per-pixel gap (P - D) / (H W) <= tol; returns xbar.
 */
static double tv_h_of(int H, int W, const double *wh, double lam, const double *x)
{
    double s = 0.0;
    for (int r = 0; r < H; ++r)
        for (int c = 0; c + 1 < W; ++c)
            s += (wh ? wh[(int64_t)r * (W - 1) + c] : lam) *
                 fabs(x[(int64_t)r * W + c + 1] - x[(int64_t)r * W + c]);
    return s;
}

static double tv_v_of(int H, int W, const double *wv, double lam, const double *x)
{
    double s = 0.0;
    for (int r = 0; r + 1 < H; ++r)
        for (int c = 0; c < W; ++c)
            s += (wv ? wv[(int64_t)r * W + c] : lam) *
                 fabs(x[(int64_t)(r + 1) * W + c] - x[(int64_t)r * W + c]);
    return s;
}

int tvo_tv2d_lagrangian(int H, int W, const double *f, const double *wh, const double *wv,
                        double lam, double tau0, int max_iters, double tol, int check_every,
                        int nthreads, double *x_out, int *iters_out, double *gap_trace)
{
    if (H < 1 || W < 1 || !f || !x_out || max_iters < 1 || !(tau0 > 0.0) || check_every < 1)
        return TVO_ERR_INVALID;
    const int64_t N = (int64_t)H * W;
    double *xh = (double *)malloc(sizeof(double) * (size_t)N);
    double *xv = (double *)malloc(sizeof(double) * (size_t)N);
    double *y = (double *)calloc((size_t)N, sizeof(double));
    double *yb = (double *)calloc((size_t)N, sizeof(double));
    double *c = (double *)malloc(sizeof(double) * (size_t)N);
    double *xr = (double *)malloc(sizeof(double) * (size_t)N);
    double *xc = (double *)malloc(sizeof(double) * (size_t)N);
    if (!xh || !xv || !y || !yb || !c || !xr || !xc) {
        free(xh); free(xv); free(y); free(yb); free(c); free(xr); free(xc);
        return TVO_ERR_NOMEM;
    }
    memcpy(xh, f, sizeof(double) * (size_t)N);
    memcpy(xv, f, sizeof(double) * (size_t)N);
    int st = TVO_OK, done = 0, k;
    for (k = 1; k <= max_iters && st == TVO_OK; ++k) {
        const double tau = tau0 / k, sigma = 1.0 / (tau * 2.0), a = 0.5 + 1.0 / tau;
        for (int64_t i = 0; i < N; ++i) c[i] = (0.5 * f[i] + (xh[i] - tau * yb[i]) / tau) / a;
        st = row_prox(H, W, c, wh, lam, a, xh, nthreads);
        if (st != TVO_OK) break;
        for (int64_t i = 0; i < N; ++i) c[i] = (0.5 * f[i] + (xv[i] + tau * yb[i]) / tau) / a;
        st = col_prox(H, W, c, wv, lam, a, xv, nthreads);
        if (st != TVO_OK) break;
        for (int64_t i = 0; i < N; ++i) {
            const double yn = y[i] + sigma * (xh[i] - xv[i]);
            yb[i] = yn + (yn - y[i]);
            y[i] = yn;
        }
        if (gap_trace) gap_trace[k - 1] = NAN;
        if (k % check_every == 0 || k == max_iters) {
            for (int64_t i = 0; i < N; ++i) x_out[i] = 0.5 * (xh[i] + xv[i]);
            const double P = tvo_rof_primal(H, W, f, wh, wv, lam, x_out);
            for (int64_t i = 0; i < N; ++i) c[i] = f[i] - 2.0 * y[i];
            st = row_prox(H, W, c, wh, lam, 0.5, xr, nthreads);
            if (st != TVO_OK) break;
            for (int64_t i = 0; i < N; ++i) c[i] = f[i] + 2.0 * y[i];
            st = col_prox(H, W, c, wv, lam, 0.5, xc, nthreads);
            if (st != TVO_OK) break;
            double D = tv_h_of(H, W, wh, lam, xr) + tv_v_of(H, W, wv, lam, xc);
            for (int64_t i = 0; i < N; ++i)
                D += 0.25 * (xr[i] - f[i]) * (xr[i] - f[i]) + xr[i] * y[i] +
                     0.25 * (xc[i] - f[i]) * (xc[i] - f[i]) - xc[i] * y[i];
            const double g = (P - D) / (double)N;
            if (gap_trace) gap_trace[k - 1] = g;
            if (tol > 0.0 && g <= tol) {
                done = 1;
                break;
            }
        }
    }
    if (iters_out) *iters_out = done ? k : (k > max_iters ? max_iters : k);
    free(xh); free(xv); free(y); free(yb); free(c); free(xr); free(xc);
    if (st != TVO_OK) return st;
    return done ? TVO_OK : TVO_NOT_CONVERGED;
}


/* ---------------- piecewise-quadratic unaries on a chain (Sec. 4.2) ----------------
 *
 * x* = argmin sum_i (a_i x_i^2/2 - b_i x_i + alpha_i |x_i - f_i|) + sum_{i<n} w_i |x_{i+1} - x_i|,
 * a_i > 0, alpha_i >= 0, w_i >= 0: the convex chain of Algorithm 2 whose unary derivatives
 * g_i(z) = a_i z - b_i + alpha_i sign(z - f_i) are piecewise linear with a jump of
 * 2 alpha_i at f_i (the piecewise-quadratic unaries of Sec. 4.2). The message (a
 * derivative) is stored explicitly, obviously rather than fast: sorted breakpoints
 * lam[0..t-1] and the linear function A_p z + B_p of every piece p = 0..t (piece p lies
 * between lam[p-1] and lam[p], with lam[-1] = -inf and lam[t] = +inf); values jump up at
 * breakpoints. The message into node 0 is 0 (one piece, A = B = 0). At node i: add g_i
 * to every piece, inserting f_i as a breakpoint; clip to [-w_i, w_i]:
 *   lambda^- = sup{z : m^_i(z) < -w_i},  lambda^+ = inf{z : m^_i(z) > w_i},
 * the new message is -w_i left of lambda^-, m^_i between, +w_i right of lambda^+; the last
 * node has w = 0 and x_{n-1} = lambda^- = lambda^+. Backward: x_i = clip(x_{i+1}, lambda^-_i,
 * lambda^+_i) (Algorithm 2).
 */
typedef struct {
    int64_t t;     /* number of breakpoints */
    double *lam;   /* breakpoints */
    double *A, *B; /* pieces 0..t */
} tvo_pwl;

/* m^ = m + g: a z - b on every piece, -alpha left of f and +alpha right of it. */
static void pq_add(tvo_pwl *h, double a, double b, double alpha, double f)
{
    int64_t pos = 0; /* pieces 0..pos lie left of f, pos+1..t right of it */
    while (pos < h->t && h->lam[pos] < f) ++pos;
    if (!(pos < h->t && h->lam[pos] == f)) {
        for (int64_t q = h->t; q > pos; --q) h->lam[q] = h->lam[q - 1];
        for (int64_t q = h->t + 1; q > pos; --q) {
            h->A[q] = h->A[q - 1];
            h->B[q] = h->B[q - 1];
        }
        h->lam[pos] = f;
        h->t += 1;
    }
    for (int64_t p = 0; p <= h->t; ++p) {
        h->A[p] += a;
        h->B[p] += -b + (p <= pos ? -alpha : alpha);
    }
}

/* Clip to [wlo, whi]; returns lambda^-, lambda^+. `o` is scratch of the same capacity. */
static void pq_clip(tvo_pwl *h, double wlo, double whi, double *lm, double *hp, tvo_pwl *o)
{
    const int64_t t = h->t;
    int64_t pl = t, pr = 0;
    double l = 0.0, r = 0.0;
    for (int64_t p = 0; p <= t; ++p) {
        const double end = (p < t) ? h->A[p] * h->lam[p] + h->B[p] : INFINITY;
        if (end >= wlo) { /* the crossing is in piece p, or at the jump into it */
            const double z = (wlo - h->B[p]) / h->A[p];
            l = (p > 0 && z < h->lam[p - 1]) ? h->lam[p - 1] : z;
            pl = p;
            break;
        }
    }
    for (int64_t p = t; p >= 0; --p) {
        const double start = (p > 0) ? h->A[p] * h->lam[p - 1] + h->B[p] : -INFINITY;
        if (start <= whi) { /* the crossing is in piece p, or at the jump out of it */
            const double z = (whi - h->B[p]) / h->A[p];
            r = (p < t && z > h->lam[p]) ? h->lam[p] : z;
            pr = p;
            break;
        }
    }
    *lm = l;
    *hp = r;
    /* breakpoints lambda^-, lam[pl..pr-1], lambda^+; pieces wlo, pl..pr, whi */
    int64_t nt = 0;
    o->lam[nt++] = l;
    o->A[0] = 0.0;
    o->B[0] = wlo;
    for (int64_t p = pl; p <= pr; ++p) {
        if (p > pl) o->lam[nt++] = h->lam[p - 1];
        o->A[nt] = h->A[p];
        o->B[nt] = h->B[p];
    }
    if (pl > pr) { /* one jump of m^ crosses both levels: lambda^- = lambda^+, a zero-length
                      piece between them at the lower level */
        o->A[nt] = 0.0;
        o->B[nt] = wlo;
    }
    o->lam[nt++] = r;
    o->A[nt] = 0.0;
    o->B[nt] = whi;
    o->t = nt;
    /* swap the buffers */
    tvo_pwl tmp = *h;
    *h = *o;
    *o = tmp;
}

static int chain_pq_core(int64_t n, const double *a, const double *b, const double *alpha,
                         const double *f, const double *w, double *x)
{
    if (n <= 0) return TVO_OK;
    const int64_t cap = 3 * n + 8;
    double *buf = (double *)malloc(sizeof(double) * (size_t)(6 * cap + 2 * n));
    if (!buf) return TVO_ERR_NOMEM;
    tvo_pwl h = {0, buf, buf + cap, buf + 2 * cap};
    tvo_pwl o = {0, buf + 3 * cap, buf + 4 * cap, buf + 5 * cap};
    double *lo = buf + 6 * cap, *hi = lo + n;
    h.A[0] = 0.0;
    h.B[0] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        pq_add(&h, a[i], b[i], alpha[i], f[i]);
        const double wi = (i < n - 1) ? w[i] : 0.0;
        pq_clip(&h, -wi, wi, &lo[i], &hi[i], &o);
    }
    x[n - 1] = 0.5 * (lo[n - 1] + hi[n - 1]);
    for (int64_t i = n - 2; i >= 0; --i) {
        double v = x[i + 1];
        if (v < lo[i]) v = lo[i];
        if (v > hi[i]) v = hi[i];
        x[i] = v;
    }
    free(buf);
    return TVO_OK;
}

/* Chains with piecewise-quadratic unaries in a CSR batch (one thread); w at a chain's
 * last node unused. */
int tvo_chain_solve_pq_batch(const double *a, const double *b, const double *alpha,
                             const double *f, const double *w, const int64_t *offsets,
                             int64_t num_chains, double *x)
{
    if (num_chains < 0 || !offsets) return TVO_ERR_INVALID;
    for (int64_t k = 0; k < num_chains; ++k) {
        const int64_t o = offsets[k], len = offsets[k + 1] - offsets[k];
        if (len < 0) return TVO_ERR_INVALID;
        for (int64_t i = 0; i < len; ++i)
            if (!(a[o + i] > 0.0) || !(alpha[o + i] >= 0.0) || (i < len - 1 && !(w[o + i] >= 0.0)))
                return TVO_ERR_INVALID;
        const int st = chain_pq_core(len, a + o, b + o, alpha + o, f + o, w + o, x + o);
        if (st != TVO_OK) return st;
    }
    return TVO_OK;
}


/* ---------------- TV-l1 denoising (Sec. 6) ----------------
 *
 * min_x TV_h(x) + TV_v(x) + sum_i |x_i - f_i|, as the saddle-point problem
 *   min_x max_y <x, y> + TV_h(x) + ||x - f||_1 - TV_v^*(y)
 * with the primal-dual iteration of eq. pd at constant steps (tau sigma = 1, theta = 1;
 * the model is not strongly convex):
 *   c = y^k / sigma + xbar^k,  y^{k+1} = sigma (c - argmin TV_v(z) + sigma/2 ||z - c||^2)
 *        (column chains, eq. prox-tv-conj)
 *   x^{k+1} = argmin TV_h(x) + ||x - f||_1 + 1/(2 tau) ||x - (x^k - tau y^{k+1})||^2
 *        (row chains with piecewise-quadratic unaries, eq. prox-pq; scaled by tau:
 *         a = 1, b = xi, alpha = tau, weights tau w_h)
 *   xbar^{k+1} = 2 x^{k+1} - x^k.
 * Start x^0 = xbar^0 = f, y^0 = 0. energy[k] = TV(x^{k+1}) + ||x^{k+1} - f||_1.
 */
static double l1_energy(int H, int W, const double *f, const double *wh, const double *wv,
                        double lam, const double *x)
{
    double s = tv_h_of(H, W, wh, lam, x) + tv_v_of(H, W, wv, lam, x);
    for (int64_t i = 0; i < (int64_t)H * W; ++i) s += fabs(x[i] - f[i]);
    return s;
}

int tvo_tv2d_l1(int H, int W, const double *f, const double *wh, const double *wv, double lam,
                double tau, int max_iters, int nthreads, double *x_out, double *energy)
{
    if (H < 1 || W < 1 || !f || !x_out || max_iters < 1 || !(tau > 0.0)) return TVO_ERR_INVALID;
    const int64_t N = (int64_t)H * W;
    const double sigma = 1.0 / tau;
    double *x = x_out;
    double *xb = (double *)malloc(sizeof(double) * (size_t)N);
    double *y = (double *)calloc((size_t)N, sizeof(double));
    double *c = (double *)malloc(sizeof(double) * (size_t)N);
    double *xh = (double *)malloc(sizeof(double) * (size_t)N);
    double *xn = (double *)malloc(sizeof(double) * (size_t)N);
    double *ones = (double *)malloc(sizeof(double) * (size_t)W);
    double *alw = (double *)malloc(sizeof(double) * (size_t)W);
    double *ww = (double *)malloc(sizeof(double) * (size_t)W);
    if (!xb || !y || !c || !xh || !xn || !ones || !alw || !ww) {
        free(xb); free(y); free(c); free(xh); free(xn); free(ones); free(alw); free(ww);
        return TVO_ERR_NOMEM;
    }
    memcpy(x, f, sizeof(double) * (size_t)N);
    memcpy(xb, f, sizeof(double) * (size_t)N);
    for (int q = 0; q < W; ++q) {
        ones[q] = 1.0;
        alw[q] = tau;
    }
    int st = TVO_OK;
    for (int k = 0; k < max_iters && st == TVO_OK; ++k) {
        for (int64_t i = 0; i < N; ++i) c[i] = y[i] / sigma + xb[i];
        st = col_prox(H, W, c, wv, lam, sigma, xh, nthreads);
        if (st != TVO_OK) break;
        for (int64_t i = 0; i < N; ++i) y[i] = sigma * (c[i] - xh[i]);
        for (int64_t i = 0; i < N; ++i) c[i] = x[i] - tau * y[i]; /* xi */
        for (int r = 0; r < H && st == TVO_OK; ++r) {
            for (int q = 0; q + 1 < W; ++q) ww[q] = tau * (wh ? wh[(int64_t)r * (W - 1) + q] : lam);
            ww[W - 1] = 0.0;
            st = chain_pq_core(W, ones, c + (int64_t)r * W, alw, f + (int64_t)r * W, ww,
                               xn + (int64_t)r * W);
        }
        if (st != TVO_OK) break;
        for (int64_t i = 0; i < N; ++i) {
            xb[i] = 2.0 * xn[i] - x[i];
            x[i] = xn[i];
        }
        if (energy) energy[k] = l1_energy(H, W, f, wh, wv, lam, x);
    }
    free(xb); free(y); free(c); free(xh); free(xn); free(ones); free(alw); free(ww);
    return st;
}


/* ---------------- non-convex chains: truncated TV, piecewise-linear unaries (Sec. 3) ----------------
 *
 * x* in argmin_x sum_i f_i(x_i) + sum_{i<n} min(w_i |x_{i+1} - x_i|, C_i),
 * f_i continuous piecewise linear (any shape, bounded below), w_i >= 0, C_i >= 0 (C_i = +inf:
 * plain TV). DP on the chain (eq. Message:update): M^_0 = f_0; M_{i,i+1} = M^_i (x) f_{i,i+1}
 * (min-convolution); M^_{i+1} = f_{i+1} + M_{i,i+1}. Messages are piecewise linear and are
 * stored as the paper's sequence (s_0, lambda_1, s_1, ..., lambda_t, s_t) together with the
 * value at lambda_1 (the sequence alone fixes a message up to a constant; the value is kept so
 * that the optimum energy can be read off). The min-convolution with min(w|z|, C) is taken as
 * three consecutive ones (Prop. ConsecutiveMinConvolution) with
 *   f^1(z) = w z for z >= 0 (+inf left of 0)   -- Algorithm 1,
 *   f^2(z) = w |z| for z <= 0 (+inf right of 0) -- Algorithm 1 on the reversed function,
 *   f^3(z) = C for z != 0, 0 at 0               -- min(h, min h + C).
 * Backward: x_{n-1} minimises M^_{n-1}; x_i = pi_{i,i+1}(x_{i+1}), pi taken from its definition
 * as an argmin of M^_i(z) + min(w_i |x_{i+1} - z|, C_i) over z (the minimum of this piecewise-
 * linear function lies at a breakpoint of M^_i, at x_{i+1}, or at x_{i+1} -+ C_i / w_i; the
 * first minimum in that order is taken), for which every M^_i is kept.
 */
typedef struct {
    int64_t t;     /* breakpoints lam[0..t-1], non-decreasing */
    double s0;     /* slope left of lam[0] */
    double *lam;
    double *s;     /* s[p]: slope right of lam[p] */
    double v0;     /* value at lam[0] (t > 0), or the constant (t = 0) */
    int64_t cap;
} tvo_plf;

static int plf_reserve(tvo_plf *h, int64_t cap)
{
    if (cap <= h->cap) return TVO_OK;
    double *l = (double *)realloc(h->lam, sizeof(double) * (size_t)cap);
    if (!l) return TVO_ERR_NOMEM;
    h->lam = l;
    double *s = (double *)realloc(h->s, sizeof(double) * (size_t)cap);
    if (!s) return TVO_ERR_NOMEM;
    h->s = s;
    h->cap = cap;
    return TVO_OK;
}

static void plf_free(tvo_plf *h)
{
    free(h->lam);
    free(h->s);
    h->lam = h->s = NULL;
    h->cap = h->t = 0;
}

/* values at the breakpoints */
static void plf_values(const tvo_plf *h, double *v)
{
    if (h->t == 0) return;
    v[0] = h->v0;
    for (int64_t p = 1; p < h->t; ++p) v[p] = v[p - 1] + h->s[p - 1] * (h->lam[p] - h->lam[p - 1]);
}

static double plf_eval(const tvo_plf *h, double z)
{
    if (h->t == 0) return h->v0;
    if (z <= h->lam[0]) return h->v0 + h->s0 * (z - h->lam[0]);
    double v = h->v0;
    int64_t p = 0;
    while (p + 1 < h->t && h->lam[p + 1] <= z) {
        v += h->s[p] * (h->lam[p + 1] - h->lam[p]);
        ++p;
    }
    return v + h->s[p] * (z - h->lam[p]);
}

static int plf_push(tvo_plf *o, double lam, double s)
{
    if (o->t == o->cap && plf_reserve(o, o->cap ? 2 * o->cap : 16) != TVO_OK) return TVO_ERR_NOMEM;
    o->lam[o->t] = lam;
    o->s[o->t] = s;
    o->t += 1;
    return TVO_OK;
}

/* eq. Message:update:a on a chain: o = h + f, breakpoints merged, slopes added. */
static int plf_sum(const tvo_plf *h, const tvo_plf *f, tvo_plf *o)
{
    o->t = 0;
    o->s0 = h->s0 + f->s0;
    int64_t i = 0, j = 0;
    while (i < h->t || j < f->t) {
        double z;
        if (j >= f->t || (i < h->t && h->lam[i] <= f->lam[j])) z = h->lam[i];
        else z = f->lam[j];
        while (i < h->t && h->lam[i] == z) ++i;
        while (j < f->t && f->lam[j] == z) ++j;
        /* slopes right of z: of the last breakpoint at or left of z in each, else s0 */
        const double sh = i > 0 ? h->s[i - 1] : h->s0;
        const double sf = j > 0 ? f->s[j - 1] : f->s0;
        if (plf_push(o, z, sh + sf) != TVO_OK) return TVO_ERR_NOMEM;
    }
    o->v0 = o->t ? plf_eval(h, o->lam[0]) + plf_eval(f, o->lam[0]) : h->v0 + f->v0;
    return TVO_OK;
}

/* h^rev(z) = h(-z): the sequence reversed and negated. */
static int plf_rev(const tvo_plf *h, tvo_plf *o)
{
    if (plf_reserve(o, h->t + 1) != TVO_OK) return TVO_ERR_NOMEM;
    o->t = h->t;
    if (h->t == 0) {
        o->s0 = -h->s0;
        o->v0 = h->v0;
        return TVO_OK;
    }
    o->s0 = -h->s[h->t - 1];
    for (int64_t k = 0; k < h->t; ++k) {
        o->lam[k] = -h->lam[h->t - 1 - k];
        o->s[k] = k + 1 < h->t ? -h->s[h->t - 2 - k] : -h->s0;
    }
    o->v0 = plf_eval(h, h->lam[h->t - 1]);
    return TVO_OK;
}

/* Algorithm 1: o = h (x) f^1 with f^1(z) = w z for z >= 0, +inf for z < 0 (h bounded below,
 * so s_0 <= 0 <= w). `v` is scratch of h->t values. */
static int plf_mc1(const tvo_plf *h, double w, tvo_plf *o, double *v)
{
    o->t = 0;
    o->s0 = h->s0;
    o->v0 = h->v0;
    const int64_t t = h->t;
    if (t == 0) return TVO_OK;
    plf_values(h, v);
    int64_t p = 0;
    while (p < t) {
        if (plf_push(o, h->lam[p], h->s[p] < w ? h->s[p] : w) != TVO_OK) return TVO_ERR_NOMEM;
        if (h->s[p] >= w) {
            /* hbar(z) = w (z - lam_p) + h(lam_p); the smallest q in p+2..t (q = t is the
             * right end, far out on the last segment) with h(lam_q) < hbar(lam_q) */
            int64_t q = p + 2;
            for (; q < t; ++q)
                if (v[q] < w * (h->lam[q] - h->lam[p]) + v[p]) break;
            if (q >= t && !(h->s[t - 1] < w)) return TVO_OK; /* [lam_p, +inf] maps to lam_p */
            if (q > t) q = t;
            /* h = hbar on the segment right of lam_{q-1} (slope s_{q-1} < w) */
            const double l0 = h->lam[q - 1];
            const double gap = v[q - 1] - (w * (l0 - h->lam[p]) + v[p]); /* >= 0 */
            const double z = l0 + gap / (w - h->s[q - 1]);
            if (plf_push(o, z, h->s[q - 1]) != TVO_OK) return TVO_ERR_NOMEM;
            p = q;
        } else {
            ++p;
        }
    }
    return TVO_OK;
}

/* o = h (x) f^3 = min(h, min h + C), C >= 0 finite; h bounded below. Drops breakpoints
 * whose two slopes agree. `v` is scratch of h->t values. */
static int plf_mc3(const tvo_plf *h, double C, tvo_plf *o, double *v)
{
    o->t = 0;
    if (h->t == 0) {
        o->s0 = h->s0;
        o->v0 = h->v0;
        return TVO_OK;
    }
    plf_values(h, v);
    double m = v[0];
    for (int64_t p = 1; p < h->t; ++p) m = v[p] < m ? v[p] : m;
    const double cap = m + C;
    /* the points (z, value) of min(h, cap), in order, then slopes between them */
    int64_t np = 0, npcap = 2 * h->t + 2;
    double *pz = (double *)malloc(sizeof(double) * (size_t)npcap);
    double *pv = (double *)malloc(sizeof(double) * (size_t)npcap);
    if (!pz || !pv) {
        free(pz);
        free(pv);
        return TVO_ERR_NOMEM;
    }
    /* left end: h rises to the left with slope -s0 >= 0 */
    double sl = h->s0;
    if (v[0] >= cap) sl = 0.0;
    else if (h->s0 < 0.0) {
        pz[np] = h->lam[0] + (cap - v[0]) / h->s0;
        pv[np++] = cap;
        sl = 0.0;
    }
    for (int64_t p = 0; p < h->t; ++p) {
        pz[np] = h->lam[p];
        pv[np++] = v[p] < cap ? v[p] : cap;
        if (p + 1 < h->t) {
            const double a = v[p] - cap, b = v[p + 1] - cap;
            if ((a < 0.0 && b > 0.0) || (a > 0.0 && b < 0.0)) {
                pz[np] = h->lam[p] + (h->lam[p + 1] - h->lam[p]) * (a / (a - b));
                pv[np++] = cap;
            }
        }
    }
    const int64_t last = h->t - 1;
    double sr = h->s[last];
    if (v[last] >= cap) sr = 0.0;
    else if (h->s[last] > 0.0) {
        pz[np] = h->lam[last] + (cap - v[last]) / h->s[last];
        pv[np++] = cap;
        sr = 0.0;
    }
    o->s0 = sl;
    o->v0 = pv[0];
    for (int64_t k = 0; k < np; ++k) {
        const double s = k + 1 < np ? (pz[k + 1] > pz[k] ? (pv[k + 1] - pv[k]) / (pz[k + 1] - pz[k])
                                                         : 0.0)
                                    : sr;
        const double s_left = o->t ? o->s[o->t - 1] : sl;
        if (k > 0 && k + 1 < np && s == s_left) continue; /* no change of slope */
        if (o->t == 0) o->v0 = pv[k];
        if (plf_push(o, pz[k], s) != TVO_OK) {
            free(pz);
            free(pv);
            return TVO_ERR_NOMEM;
        }
    }
    free(pz);
    free(pv);
    return TVO_OK;
}

/* the objective of the backward step at z */
static double nc_back_obj(const tvo_plf *h, double z, double xn, double w, double C)
{
    double d = w * fabs(xn - z);
    if (d > C) d = C;
    return plf_eval(h, z) + d;
}

/*
 * One chain of n nodes. Unary i: breakpoints ul[uo[i]..uo[i+1]), values uv there, slopes
 * sl[i] (left end) and sr[i] (right end). w[i], C[i]: edge (i, i+1) (entries at i = n-1
 * unused; C = INFINITY for plain TV). x: n outputs; *energy: the optimum.
 */
static int chain_nonconvex_core(int64_t n, const int64_t *uo, const double *ul, const double *uv,
                                const double *sl, const double *sr, const double *w,
                                const double *C, double *x, double *energy)
{
    if (n <= 0) {
        *energy = 0.0;
        return TVO_OK;
    }
    tvo_plf *Mh = (tvo_plf *)calloc((size_t)n, sizeof(tvo_plf)); /* M^_i, kept */
    tvo_plf f = {0}, a = {0}, b = {0};
    double *v = NULL;
    int64_t vcap = 0;
    int st = TVO_OK;
    if (!Mh) return TVO_ERR_NOMEM;
    for (int64_t i = 0; i < n && st == TVO_OK; ++i) {
        /* f_i as a sequence */
        const int64_t t = uo[i + 1] - uo[i];
        st = plf_reserve(&f, t + 1);
        if (st != TVO_OK) break;
        f.t = t;
        if (t == 0) {
            /* bounded below and linear: a constant */
            f.s0 = 0.0;
            f.v0 = 0.0;
        } else {
            f.s0 = sl[i];
            f.v0 = uv[uo[i]];
            for (int64_t p = 0; p < t; ++p) {
                f.lam[p] = ul[uo[i] + p];
                f.s[p] = p + 1 < t ? (ul[uo[i] + p + 1] > ul[uo[i] + p]
                                          ? (uv[uo[i] + p + 1] - uv[uo[i] + p]) /
                                                (ul[uo[i] + p + 1] - ul[uo[i] + p])
                                          : 0.0)
                                   : sr[i];
            }
        }
        if (i == 0) {
            st = plf_reserve(&Mh[0], t + 1);
            if (st != TVO_OK) break;
            Mh[0].t = f.t;
            Mh[0].s0 = f.s0;
            Mh[0].v0 = f.v0;
            memcpy(Mh[0].lam, f.lam, sizeof(double) * (size_t)t);
            memcpy(Mh[0].s, f.s, sizeof(double) * (size_t)t);
        } else {
            st = plf_sum(&b, &f, &Mh[i]); /* b holds M_{i-1,i} */
            if (st != TVO_OK) break;
        }
        if (i == n - 1) break;
        /* M_{i,i+1} = ((M^_i (x) f^1) (x) f^2) (x) f^3 */
        const tvo_plf *h = &Mh[i];
        const int64_t need = 2 * h->t + 4;
        if (need > vcap) {
            double *nv = (double *)realloc(v, sizeof(double) * (size_t)need);
            if (!nv) {
                st = TVO_ERR_NOMEM;
                break;
            }
            v = nv;
            vcap = need;
        }
        if ((st = plf_mc1(h, w[i], &a, v)) != TVO_OK) break;       /* (x) f^1 */
        if ((st = plf_rev(&a, &b)) != TVO_OK) break;
        if ((st = plf_mc1(&b, w[i], &a, v)) != TVO_OK) break;      /* (x) f^2 via reversal */
        if ((st = plf_rev(&a, &b)) != TVO_OK) break;
        if (isfinite(C[i])) {
            if (2 * b.t + 4 > vcap) {
                double *nv = (double *)realloc(v, sizeof(double) * (size_t)(2 * b.t + 4));
                if (!nv) {
                    st = TVO_ERR_NOMEM;
                    break;
                }
                v = nv;
                vcap = 2 * b.t + 4;
            }
            if ((st = plf_mc3(&b, C[i], &a, v)) != TVO_OK) break;  /* (x) f^3 */
            if ((st = plf_reserve(&b, a.t + 1)) != TVO_OK) break;
            b.t = a.t;
            b.s0 = a.s0;
            b.v0 = a.v0;
            memcpy(b.lam, a.lam, sizeof(double) * (size_t)a.t);
            memcpy(b.s, a.s, sizeof(double) * (size_t)a.t);
        }
    }
    if (st == TVO_OK) {
        /* x_{n-1}: the first minimiser of M^_{n-1} among its breakpoints */
        const tvo_plf *h = &Mh[n - 1];
        double best = h->v0, bz = h->t ? h->lam[0] : 0.0, val = h->v0;
        for (int64_t p = 1; p < h->t; ++p) {
            val += h->s[p - 1] * (h->lam[p] - h->lam[p - 1]);
            if (val < best) {
                best = val;
                bz = h->lam[p];
            }
        }
        x[n - 1] = bz;
        *energy = best;
        for (int64_t i = n - 2; i >= 0; --i) {
            const tvo_plf *g = &Mh[i];
            const double xn = x[i + 1];
            double bzz = xn, bo = nc_back_obj(g, xn, xn, w[i], C[i]);
            for (int64_t p = 0; p < g->t; ++p) {
                const double o = nc_back_obj(g, g->lam[p], xn, w[i], C[i]);
                if (o < bo) {
                    bo = o;
                    bzz = g->lam[p];
                }
            }
            if (isfinite(C[i]) && w[i] > 0.0) {
                const double r = C[i] / w[i];
                const double zc[2] = {xn - r, xn + r};
                for (int k = 0; k < 2; ++k) {
                    const double o = nc_back_obj(g, zc[k], xn, w[i], C[i]);
                    if (o < bo) {
                        bo = o;
                        bzz = zc[k];
                    }
                }
            }
            x[i] = bzz;
        }
    }
    for (int64_t i = 0; i < n; ++i) plf_free(&Mh[i]);
    free(Mh);
    plf_free(&f);
    plf_free(&a);
    plf_free(&b);
    free(v);
    return st;
}

/* Batch of contiguous chains (CSR offsets over nodes). uo: node -> breakpoint offsets
 * (N + 1 entries, absolute). energy: one per chain. */
int tvo_chain_solve_nonconvex_batch(const int64_t *uo, const double *ul, const double *uv,
                                    const double *sl, const double *sr, const double *w,
                                    const double *C, const int64_t *offsets, int64_t nchains,
                                    double *x, double *energy)
{
    if (!uo || !offsets || !x || !energy || nchains < 0) return TVO_ERR_INVALID;
    for (int64_t k = 0; k < nchains; ++k) {
        const int64_t o = offsets[k], len = offsets[k + 1] - o;
        if (len < 0) return TVO_ERR_INVALID;
        for (int64_t i = 0; i < len; ++i)
            if (uo[o + i + 1] < uo[o + i]) return TVO_ERR_INVALID;
        const int st = chain_nonconvex_core(len, uo + o, ul, uv, sl + o, sr + o, w + o, C + o,
                                            x + o, &energy[k]);
        if (st != TVO_OK) return st;
    }
    return TVO_OK;
}
