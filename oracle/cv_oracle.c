/*
 * cv_oracle.c -- plain FP64 CPU oracle for the Clip-and-Verify hot path
 * (arXiv 2512.11087, "Clip-and-Verify: linear constraint-driven domain clipping").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py load this library.  The product path
 * (the CUDA library behind include/clipverify.h) never calls, links or includes it,
 * and this file includes nothing from the product.
 *
 * Everything is computed in double precision with straightforward loops in the
 * order the paper states the steps; there is no blocking or fusion.  The only
 * library primitive used is qsort (the argsort of Algorithm 1).
 *
 * Network: L affine layers z^(i) = W^(i) zhat^(i-1) + b^(i), zhat^(0) = x,
 * zhat^(i) = ReLU(z^(i)) for the hidden layers i = 1..L-1, output y = z^(L).
 * Weights are passed concatenated: W^(i) is dims[i] x dims[i-1] row-major.
 * Hidden neurons get a global id: hoff[i] + j for neuron j of hidden layer i.
 *
 * Conventions fixed where the paper leaves room (readings of the paper, not its words):
 *  - every linear constraint is a row  g.x + h <= 0  (Theorem 2 and Algorithm 2's update);
 *  - an activation split  z_j >= 0  gives the row  -Abar_j.x - cbar_j <= 0,  a split
 *    z_j <= 0  gives  Aund_j.x + cund_j <= 0  (Section 3.4, "validate" implication);
 *  - the unstable lower slope alpha defaults to the adaptive rule alpha = [u >= -l];
 *  - stability and feasibility use the paper's thresholds exactly: active iff l >= 0,
 *    inactive iff u <= 0 (Lemma, ReLU relaxation), a row is infeasible iff its box
 *    minimum is > 0 and redundant iff its box maximum is <= 0;
 *  - the clipped input box is stored in FP32 (the interface format), each bound
 *    rounded outward, and the later steps use that stored box;
 *  - Algorithm 1's partial multiplier sum excludes row k (the text of Section 3.2);
 *    the supergradient is non-increasing and i* ranges over 0..n with q_(0) = -inf.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* network indexing                                                          */
/* ------------------------------------------------------------------------- */
typedef struct {
    int L;
    const int* dims;          /* dims[0..L] */
    const double* W;          /* concatenated W^(1..L) */
    const double* b;          /* concatenated b^(1..L) */
    long woff[64];            /* woff[i]: start of W^(i) */
    long boff[64];            /* boff[i]: start of b^(i) */
    int hoff[64];             /* hoff[i]: first global id of hidden layer i */
    int H;                    /* number of hidden neurons */
} net_t;

static int net_init(net_t* n, int L, const int* dims, const double* W, const double* b) {
    if (L < 1 || L > 62) return -1;
    n->L = L; n->dims = dims; n->W = W; n->b = b;
    long wo = 0, bo = 0; int ho = 0;
    for (int i = 1; i <= L; ++i) {
        n->woff[i] = wo; n->boff[i] = bo;
        wo += (long)dims[i] * dims[i - 1];
        bo += dims[i];
        n->hoff[i] = ho;
        if (i < L) ho += dims[i];
    }
    n->H = ho;
    return 0;
}
static inline const double* Wl(const net_t* n, int i) { return n->W + n->woff[i]; }
static inline const double* bl(const net_t* n, int i) { return n->b + n->boff[i]; }

/* outward rounding of a double onto the FP32 grid */
static double rdown32(double x) {
    if (isinf(x) || isnan(x)) return x;
    float f = (float)x;
    if ((double)f > x) f = nextafterf(f, -INFINITY);
    return (double)f;
}
static double rup32(double x) {
    if (isinf(x) || isnan(x)) return x;
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return (double)f;
}

/* ------------------------------------------------------------------------- */
/* Lemma A.1 (dual-norm concretization over a box):                          */
/*   min_{x in box} a.x + c = a.xhat - |a|.eps + c,  max = a.xhat + |a|.eps + c */
/* ------------------------------------------------------------------------- */
void orc_concretize(int n, const double* a, double c, const double* lo, const double* hi,
                    double* vmin, double* vmax) {
    double s = 0.0, r = 0.0;
    for (int j = 0; j < n; ++j) {
        double xh = 0.5 * (lo[j] + hi[j]);
        double ep = 0.5 * (hi[j] - lo[j]);
        s += a[j] * xh;
        r += fabs(a[j]) * ep;
    }
    if (vmin) *vmin = s - r + c;
    if (vmax) *vmax = s + r + c;
}

/* ------------------------------------------------------------------------- */
/* Lemma (relaxation of a ReLU layer in CROWN), Appendix "Formulating        */
/* Bounding Hyperplanes": the diagonal entry D_jj and offset for coefficient */
/* p on relu(z_j), z_j in [l, u].                                            */
/*   state +1 (l >= 0): D = 1, offset 0;  state -1 (u <= 0): D = 0, offset 0 */
/*   unstable, p >= 0: D = alpha, offset 0                                   */
/*   unstable, p <  0: D = u/(u-l), offset -u l/(u-l)                        */
/* ------------------------------------------------------------------------- */
static void relu_relax(double p, double l, double u, int state, double alpha,
                       double* d, double* e) {
    if (state > 0) { *d = 1.0; *e = 0.0; return; }
    if (state < 0) { *d = 0.0; *e = 0.0; return; }
    if (p >= 0.0) { *d = alpha; *e = 0.0; return; }
    double s = u / (u - l);
    *d = s;
    *e = -s * l;
}

/* adaptive lower slope (default reading of "fixed or optimized" alpha) */
static double alpha_rule(int mode, double l, double u) {
    if (mode == 1) return 1.0;
    if (mode == 2) return 0.0;
    return (u >= -l) ? 1.0 : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Back-substitution (the Omega recursion of the Appendix): starting from     */
/*   f >= Lam . z^(k) + bias   (Lam: rows x dims[k])                          */
/* substitute z^(i) = W^(i) zhat^(i-1) + b^(i) and relax zhat^(i-1) layer by  */
/* layer down to the input, giving  f >= Lam0 . x + bias.                     */
/* hl/hu/hstate give the bounds and stability of every hidden neuron.        */
/* alpha (rows x H, may be NULL) gives per-row lower slopes.                  */
/* If scale != NULL it accumulates the magnitude scale                        */
/*   sum_i |Lam^(i)| (|W^(i)| zmag^(i-1) + |b^(i)|)                           */
/* with zmag the given magnitude bound of every hidden neuron (used only to  */
/* state the tolerance of the CUDA comparison).  If keepP != NULL, the        */
/* products P^(i) = Lam^(i) W^(i) for i = 2..k are saved (for the adjoint).   */
/* ------------------------------------------------------------------------- */
static void backward_beta(const net_t* n, int k, int rows, const double* Lam_k,
                          const double* hl, const double* hu, const signed char* hstate,
                          const double* alpha, int alpha_mode,
                          double* Lam0, double* bias,
                          double* scale, const double* zmag, const double* xmag,
                          double** keepP, const double* beta, const signed char* bsign);
static void backward(const net_t* n, int k, int rows, const double* Lam_k,
                     const double* hl, const double* hu, const signed char* hstate,
                     const double* alpha, int alpha_mode,
                     double* Lam0, double* bias,
                     double* scale, const double* zmag, const double* xmag,
                     double** keepP) {
    backward_beta(n, k, rows, Lam_k, hl, hu, hstate, alpha, alpha_mode, Lam0, bias, scale, zmag, xmag, keepP,
                  NULL, NULL);
}

/* The same with split multipliers (the beta-CROWN form of the split constraints of Section 3.4):  */
/* beta [rows x H] >= 0 and bsign [H] (+1: split z_g >= 0, -1: z_g <= 0, 0: none).  A split holds   */
/* the constraint -bsign_g z_g <= 0, so adding beta_g (-bsign_g z_g) to the bound keeps it a lower   */
/* bound on the subdomain: after hidden layer i-1's relaxation, Lam_g -= bsign_g beta_g.            */
static void backward_beta(const net_t* n, int k, int rows, const double* Lam_k,
                          const double* hl, const double* hu, const signed char* hstate,
                          const double* alpha, int alpha_mode,
                          double* Lam0, double* bias,
                          double* scale, const double* zmag, const double* xmag,
                          double** keepP, const double* beta, const signed char* bsign) {
    const int* d = n->dims;
    int wmax = 0;
    for (int i = 0; i <= n->L; ++i) if (d[i] > wmax) wmax = d[i];
    double* cur = (double*)malloc(sizeof(double) * (size_t)rows * wmax);
    double* nxt = (double*)malloc(sizeof(double) * (size_t)rows * wmax);
    double* V = (double*)malloc(sizeof(double) * wmax);
    memcpy(cur, Lam_k, sizeof(double) * (size_t)rows * d[k]);
    for (int i = k; i >= 1; --i) {
        const double* W = Wl(n, i);
        const double* bb = bl(n, i);
        int no = d[i], ni = d[i - 1];
        if (scale) {
            for (int j = 0; j < no; ++j) {
                double v = fabs(bb[j]);
                for (int q = 0; q < ni; ++q) {
                    double zm = (i == 1) ? xmag[q] : zmag[n->hoff[i - 1] + q];
                    v += fabs(W[(long)j * ni + q]) * zm;
                }
                V[j] = v;
            }
        }
        /* rows are independent: threads over rows (single-threaded inside the per-subdomain loop) */
#pragma omp parallel for schedule(static) if (rows >= 64)
        for (int r = 0; r < rows; ++r) {
            const double* lam = cur + (long)r * no;
            double* P = nxt + (long)r * ni;
            double bsum = 0.0, ssum = 0.0;
            for (int j = 0; j < no; ++j) {
                bsum += lam[j] * bb[j];
                if (scale) ssum += fabs(lam[j]) * V[j];
            }
            bias[r] += bsum;
            if (scale) scale[r] += ssum;
            /* P_q = sum_j lam_j W_jq, each sum taken over j in increasing order (the j loop outside
               only makes the reads of W row-wise; every P_q sees the same additions in the same order) */
            for (int q = 0; q < ni; ++q) P[q] = 0.0;
            for (int j = 0; j < no; ++j) {
                const double lj = lam[j];
                if (lj == 0.0) continue;  /* a zero term adds nothing (inactive neurons, identity starts) */
                const double* w = W + (long)j * ni;
                for (int q = 0; q < ni; ++q) P[q] += lj * w[q];
            }
        }
        if (i == 1) {
            memcpy(Lam0, nxt, sizeof(double) * (size_t)rows * ni);
            break;
        }
        if (keepP) memcpy(keepP[i], nxt, sizeof(double) * (size_t)rows * ni);
        /* relax hidden layer i-1 */
        int ho = n->hoff[i - 1];
        for (int r = 0; r < rows; ++r) {
            double* P = nxt + (long)r * ni;
            double* out = cur + (long)r * ni;
            double bsum = 0.0;
            for (int q = 0; q < ni; ++q) {
                int g = ho + q;
                double a = alpha ? alpha[(long)r * n->H + g] : alpha_rule(alpha_mode, hl[g], hu[g]);
                double dd, ee;
                relu_relax(P[q], hl[g], hu[g], hstate[g], a, &dd, &ee);
                out[q] = P[q] * dd;
                if (beta && bsign[g]) out[q] -= (double)bsign[g] * beta[(long)r * n->H + g];
                bsum += P[q] * ee;
            }
            bias[r] += bsum;
        }
    }
    free(cur); free(nxt); free(V);
}

/* stability of a neuron from its bounds (the three cases of the ReLU Lemma) */
static signed char stab_state(double l, double u) {
    if (l >= 0.0) return 1;
    if (u <= 0.0) return -1;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Root cache (Get_Constraints of Algorithm 5; Section 3.4 "cache and reuse"): */
/* CROWN over every hidden layer in turn.  For layer k the lower planes are   */
/* obtained by back-substituting Lam = I, the upper planes by Lam = -I (the   */
/* lower bound of -z), both with the relaxations of layers < k.  Bounds are   */
/* their concretizations over the root box (Lemma A.1).                       */
/* Outputs: l,u [H]; planes lA,uA [H x n0], lc,uc [H]; pscale [H] =          */
/* |A| max(|lo|,|hi|) + |c| (max over the two planes, the magnitude scale of  */
/* the neuron's concretization); bscale [H] (may be NULL): the magnitude of   */
/* every term of the back-substitution that formed the bound,                 */
/* sum_i |Lam^(i)|(|W^(i)| zmag^(i-1) + |b^(i)|) + |A| xmag + |c|.            */
/* ------------------------------------------------------------------------- */
int orc_root_crown(int L, const int* dims, const double* W, const double* b,
                   const double* lo, const double* hi, int alpha_mode,
                   double* l_all, double* u_all, double* lA, double* lc,
                   double* uA, double* uc, double* pscale, double* bscale) {
    net_t n;
    if (net_init(&n, L, dims, W, b)) return -1;
    int n0 = dims[0];
    signed char* st = (signed char*)calloc((size_t)n.H + 1, 1);
    double* zmag = (double*)calloc((size_t)n.H + 1, sizeof(double));
    double* xmag = (double*)malloc(sizeof(double) * n0);
    for (int q = 0; q < n0; ++q) xmag[q] = fmax(fabs(lo[q]), fabs(hi[q]));
    for (int k = 1; k <= L - 1; ++k) {
        int nk = dims[k];
        int ho = n.hoff[k];
        double* Lam = (double*)calloc((size_t)nk * nk, sizeof(double));
        double* bias = (double*)calloc(nk, sizeof(double));
        double* s1 = (double*)calloc(nk, sizeof(double));
        double* s2 = (double*)calloc(nk, sizeof(double));
        /* lower planes */
        for (int j = 0; j < nk; ++j) Lam[(long)j * nk + j] = 1.0;
        backward(&n, k, nk, Lam, l_all, u_all, st, NULL, alpha_mode,
                 lA + (long)ho * n0, bias, s1, zmag, xmag, NULL);
        for (int j = 0; j < nk; ++j) lc[ho + j] = bias[j];
        /* upper planes: lower bound of -z, negated */
        memset(Lam, 0, sizeof(double) * (size_t)nk * nk);
        memset(bias, 0, sizeof(double) * nk);
        for (int j = 0; j < nk; ++j) Lam[(long)j * nk + j] = -1.0;
        backward(&n, k, nk, Lam, l_all, u_all, st, NULL, alpha_mode,
                 uA + (long)ho * n0, bias, s2, zmag, xmag, NULL);
        for (int j = 0; j < nk; ++j) {
            double* a = uA + (long)(ho + j) * n0;
            for (int q = 0; q < n0; ++q) a[q] = -a[q];
            uc[ho + j] = -bias[j];
        }
        for (int j = 0; j < nk; ++j) {
            int g = ho + j;
            double vmin, vmax, dum;
            orc_concretize(n0, lA + (long)g * n0, lc[g], lo, hi, &vmin, &dum);
            orc_concretize(n0, uA + (long)g * n0, uc[g], lo, hi, &dum, &vmax);
            l_all[g] = vmin;
            u_all[g] = vmax;
            double p1 = fabs(lc[g]), p2 = fabs(uc[g]);
            for (int q = 0; q < n0; ++q) {
                double xm = fmax(fabs(lo[q]), fabs(hi[q]));
                p1 += fabs(lA[(long)g * n0 + q]) * xm;
                p2 += fabs(uA[(long)g * n0 + q]) * xm;
            }
            pscale[g] = fmax(p1, p2);
            st[g] = stab_state(vmin, vmax);
            zmag[g] = fmax(fabs(vmin), fabs(vmax));
        }
        /* back-substitution magnitude scale: sum_i |Lam^(i)| V^(i) + |Lam_0| xmag + |c| */
        for (int j = 0; j < nk; ++j) {
            int g = ho + j;
            double t1 = s1[j] + fabs(lc[g]), t2 = s2[j] + fabs(uc[g]);
            for (int q = 0; q < n0; ++q) {
                t1 += fabs(lA[(long)g * n0 + q]) * xmag[q];
                t2 += fabs(uA[(long)g * n0 + q]) * xmag[q];
            }
            if (bscale) bscale[g] = fmax(t1, t2);
        }
        free(Lam); free(bias); free(s1); free(s2);
    }
    free(st); free(zmag); free(xmag);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Row pre-check (Section 3.2 a-priori infeasibility; Appendix D.3 redundancy) */
/*   v_min = min_box g.x + h,  v_max = max_box g.x + h  (Lemma A.1)           */
/*   infeasible iff v_min > 0;  redundant iff v_max <= 0                      */
/*   s = sum |g| max(|lo|,|hi|) + |h|  (magnitude scale, reported only)       */
/* return: 1 infeasible, 2 redundant, 0 active                                */
/* ------------------------------------------------------------------------- */
int orc_row_check(int n, const double* g, double h, const double* lo, const double* hi,
                  double* vmin, double* vmax, double* s_out) {
    double a, bmax, s = fabs(h);
    orc_concretize(n, g, h, lo, hi, &a, &bmax);
    for (int j = 0; j < n; ++j) s += fabs(g[j]) * fmax(fabs(lo[j]), fabs(hi[j]));
    if (vmin) *vmin = a;
    if (vmax) *vmax = bmax;
    if (s_out) *s_out = s;
    if (a > 0.0) return 1;
    if (bmax <= 0.0) return 2;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Theorem 2 / Algorithm 2 (relaxed clipping, parallel): every row is applied */
/* to the SAME input box; per coordinate i with g_i != 0                      */
/*   x_i^clip = (-sum_{j!=i}(g_j xhat_j - |g_j| eps_j) - h) / g_i             */
/*   g_i > 0: hi'_i = min(hi'_i, x_i^clip);  g_i < 0: lo'_i = max(lo'_i, x_i^clip) */
/* Rows flagged infeasible/redundant by the pre-check are skipped by the      */
/* caller.  Results stay in FP64 here; the caller rounds outward.             */
/* ------------------------------------------------------------------------- */
void orc_relaxed_clip_row(int n, const double* g, double h, const double* lo, const double* hi,
                          double* lo_new, double* hi_new) {
    for (int i = 0; i < n; ++i) {
        if (g[i] == 0.0) continue;
        double s = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double xh = 0.5 * (lo[j] + hi[j]);
            double ep = 0.5 * (hi[j] - lo[j]);
            s += g[j] * xh - fabs(g[j]) * ep;
        }
        double xc = (-s - h) / g[i];
        if (g[i] > 0.0) { if (xc < hi_new[i]) hi_new[i] = xc; }
        else            { if (xc > lo_new[i]) lo_new[i] = xc; }
    }
}

/* Algorithm 2 over R rows (rows = R x n, h = R).  Returns 1 if the clipped   */
/* box is empty (some lo' > hi').  Pre-check flags are applied inside.        */
int orc_relaxed_clip_parallel(int n, int R, const double* G, const double* h,
                              const double* lo, const double* hi,
                              double* lo_new, double* hi_new) {
    for (int i = 0; i < n; ++i) { lo_new[i] = lo[i]; hi_new[i] = hi[i]; }
    int infeas = 0;
    for (int k = 0; k < R; ++k) {
        int f = orc_row_check(n, G + (long)k * n, h[k], lo, hi, NULL, NULL, NULL);
        if (f == 1) infeas = 1;
        if (f != 0) continue;
        orc_relaxed_clip_row(n, G + (long)k * n, h[k], lo, hi, lo_new, hi_new);
    }
    for (int i = 0; i < n; ++i) if (lo_new[i] > hi_new[i]) infeas = 1;
    return infeas;
}

/* Algorithm 3 (relaxed clipping, sequential): the box centre and radius are  */
/* recomputed after each row (Appendix "Sequential Clipping").                */
int orc_relaxed_clip_sequential(int n, int R, const double* G, const double* h,
                                const double* lo, const double* hi,
                                double* lo_new, double* hi_new) {
    double* clo = (double*)malloc(sizeof(double) * n);
    double* chi = (double*)malloc(sizeof(double) * n);
    for (int i = 0; i < n; ++i) { clo[i] = lo[i]; chi[i] = hi[i]; }
    int infeas = 0;
    for (int k = 0; k < R && !infeas; ++k) {
        int f = orc_row_check(n, G + (long)k * n, h[k], clo, chi, NULL, NULL, NULL);
        if (f == 1) { infeas = 1; break; }
        if (f != 0) continue;
        for (int i = 0; i < n; ++i) { lo_new[i] = clo[i]; hi_new[i] = chi[i]; }
        orc_relaxed_clip_row(n, G + (long)k * n, h[k], clo, chi, lo_new, hi_new);
        for (int i = 0; i < n; ++i) {
            clo[i] = fmax(clo[i], lo_new[i]);
            chi[i] = fmin(chi[i], hi_new[i]);
            if (clo[i] > chi[i]) infeas = 1;
        }
    }
    for (int i = 0; i < n; ++i) { lo_new[i] = clo[i]; hi_new[i] = chi[i]; }
    free(clo); free(chi);
    return infeas;
}

/* ------------------------------------------------------------------------- */
/* Constraint importance heuristic (Appendix, details of heuristics): for the  */
/* box centre xhat, the distance of row k's hyperplane g.x + h = 0 is          */
/*   d_k = |g_k.xhat + h_k| / ||g_k||_2   (+inf for a zero row),               */
/* and the rows are taken in ascending d (equal distances keep their order).   */
/* perm receives the row indices in that order.                                */
/* ------------------------------------------------------------------------- */
void orc_row_order(int n, int R, const double* G, const double* h, const double* lo,
                   const double* hi, int* perm) {
    double* d = (double*)malloc(sizeof(double) * (R > 0 ? R : 1));
    for (int k = 0; k < R; ++k) {
        const double* g = G + (long)k * n;
        double s = h[k], nn = 0.0;
        for (int j = 0; j < n; ++j) {
            s += g[j] * 0.5 * (lo[j] + hi[j]);
            nn += g[j] * g[j];
        }
        d[k] = nn > 0.0 ? fabs(s) / sqrt(nn) : INFINITY;
        perm[k] = k;
    }
    /* insertion sort: stable */
    for (int a = 1; a < R; ++a) {
        int p = perm[a], b = a - 1;
        while (b >= 0 && d[perm[b]] > d[p]) { perm[b + 1] = perm[b]; --b; }
        perm[b + 1] = p;
    }
    free(d);
}

/* ------------------------------------------------------------------------- */
/* Input BaB split step (Algorithm 4: Domain_Filter, then Batch_Split with the */
/* parent's hyperplanes shared by both children; Section 3.3, final-layer     */
/* bounds as constraints).  Parents verified or infeasible are dropped.  For  */
/* each kept parent b, in order, with U = { r : lower_r <= 0 } its unproven  */
/* spec rows:                                                                 */
/*   axis = argmax_i (hi_i - lo_i) * sum_{r in U} |A_r,i|  (FP32, r ascending; */
/*          the first maximum; the widest axis when every score is 0)         */
/*   mid  = fl(fl(lo + hi) * 0.5)  on that axis (FP32)                       */
/*   children [lo, mid] and [mid, hi] on the axis, the parent's box elsewhere */
/*   |U| = 1: each child gets the row  A_r.x + c_r <= 0  (the only part of    */
/*            the parent where f_r may still be <= 0); otherwise no row.     */
/* The arithmetic is FP32 on purpose: the GPU takes the same decisions in the */
/* same precision.  Returns the number of children (2K).                      */
/* ------------------------------------------------------------------------- */
int orc_input_split(int B, int n0, int m, const float* lo, const float* hi, const float* A, const float* c,
                    const float* lower, const unsigned char* verified, const unsigned char* infeasible,
                    float* lo_out, float* hi_out, int* row_off, float* G, float* h, int* parent) {
    int K = 0, nr = 0;
    row_off[0] = 0;
    for (int b = 0; b < B; ++b) {
        if (verified[b] || infeasible[b]) continue;
        const float* l = lo + (long)b * n0;
        const float* u = hi + (long)b * n0;
        int nun = 0, r1 = -1;
        for (int r = 0; r < m; ++r)
            if (!(lower[(long)b * m + r] > 0.0f)) { ++nun; r1 = r; }
        int ax = 0;
        float best = -1.0f;
        for (int i = 0; i < n0; ++i) {
            float w = u[i] - l[i];
            float sc = 0.0f;
            for (int r = 0; r < m; ++r)
                if (!(lower[(long)b * m + r] > 0.0f)) sc += fabsf(A[((long)b * m + r) * n0 + i]);
            float score = w * sc;
            if (score > best) { best = score; ax = i; }
        }
        if (!(best > 0.0f)) {
            best = -1.0f;
            for (int i = 0; i < n0; ++i) {
                float w = u[i] - l[i];
                if (w > best) { best = w; ax = i; }
            }
        }
        float sum = l[ax] + u[ax];
        float mid = sum * 0.5f;
        for (int k = 0; k < 2; ++k) {
            int ch = 2 * K + k;
            float* lo2 = lo_out + (long)ch * n0;
            float* hi2 = hi_out + (long)ch * n0;
            for (int i = 0; i < n0; ++i) { lo2[i] = l[i]; hi2[i] = u[i]; }
            if (k == 0) hi2[ax] = mid; else lo2[ax] = mid;
            if (nun == 1) {
                for (int i = 0; i < n0; ++i) G[(long)nr * n0 + i] = A[((long)b * m + r1) * n0 + i];
                h[nr] = c[(long)b * m + r1];
                ++nr;
            }
            row_off[ch + 1] = nr;
            parent[ch] = b;
        }
        ++K;
    }
    return 2 * K;
}

/* ------------------------------------------------------------------------- */
/* BaBSR intercept score of a cached neuron (Appendix, neuron selection       */
/* heuristic): for an unstable neuron (mask 0, l < 0 < u)                     */
/*   score = max(0,-l) max(0,u) / (u - l) * w,  w = max(0, -weight) or 1      */
/* (the intercept of the upper ReLU line times the weight of the neuron in    */
/* the bound); -1 for any other neuron.  FP32, in this order, so that the GPU */
/* takes the same decisions.                                                  */
/* ------------------------------------------------------------------------- */
static float babsr_score(float l, float u, signed char mask, const float* weight, long o) {
    if (mask != 0 || !(l < 0.0f) || !(u > 0.0f)) return -1.0f;
    float p = fmaxf(0.0f, -l) * fmaxf(0.0f, u);
    float s = p / (u - l);
    if (weight) s = s * fmaxf(0.0f, -weight[o]);
    return s;
}

/* Activation BaB split step (Algorithm 5: Domain_Filter, Batch_Split on one  */
/* ReLU).  Verified or infeasible parents are dropped; a kept parent branches */
/* on its highest-scoring unstable cached neuron (the first slot among equal  */
/* scores); child 2k gets the split z <= 0 (code -(id+1)), child 2k+1 z >= 0  */
/* (+(id+1)), after the parent's own codes; both inherit the parent's box and */
/* cached bounds.  A kept parent with no unstable cached neuron gets no       */
/* children and stuck[b] = 1.  Returns the number of children.                */
int orc_activation_split(int B, int U, int n0, const int* ids, const int* split_off, const int* split_ids,
                         const float* lo, const float* hi, const float* l, const float* u,
                         const signed char* mask, const float* weight, const unsigned char* verified,
                         const unsigned char* infeasible, int* split_off_out, int* split_ids_out,
                         float* lo_out, float* hi_out, float* l_out, float* u_out, int* parent, int* branched,
                         unsigned char* stuck) {
    int n = 0, ns = 0;
    split_off_out[0] = 0;
    for (int b = 0; b < B; ++b) {
        stuck[b] = 0;
        if (verified[b] || infeasible[b]) continue;
        int best = -1;
        float bs = -1.0f;
        for (int c = 0; c < U; ++c) {
            long o = (long)b * U + c;
            float sc = babsr_score(l[o], u[o], mask[o], weight, o);
            if (sc > bs) { bs = sc; best = c; }  /* unstable scores are >= 0 > -1: the first maximum */
        }
        if (best < 0) { stuck[b] = 1; continue; }
        int k0 = split_off ? split_off[b] : 0, k1 = split_off ? split_off[b + 1] : 0;
        for (int side = 0; side < 2; ++side) {
            for (int q = k0; q < k1; ++q) split_ids_out[ns++] = split_ids[q];
            split_ids_out[ns++] = side ? ids[best] + 1 : -(ids[best] + 1);
            split_off_out[n + 1] = ns;
            memcpy(lo_out + (long)n * n0, lo + (long)b * n0, sizeof(float) * n0);
            memcpy(hi_out + (long)n * n0, hi + (long)b * n0, sizeof(float) * n0);
            memcpy(l_out + (long)n * U, l + (long)b * U, sizeof(float) * U);
            memcpy(u_out + (long)n * U, u + (long)b * U, sizeof(float) * U);
            parent[n] = b;
            branched[n] = best;
            ++n;
        }
    }
    return n;
}

/* Top-k targets for complete clipping (Algorithms 4/5 Top-K_Heuristic with  */
/* the BaBSR score): per subdomain and hidden layer, the k unstable cached     */
/* neurons of highest score (a neuron outranks another with a higher score,   */
/* or an equal one and a lower slot), listed in slot order as a CSR of slots. */
/* layer_of[c]: the hidden layer of slot c.  Returns the number of entries.   */
int orc_select_targets(int B, int U, const int* layer_of, const float* l, const float* u, const signed char* mask,
                       const float* weight, int k, int* tgt_off, int* tgt_ids) {
    int n = 0;
    tgt_off[0] = 0;
    for (int b = 0; b < B; ++b) {
        for (int c = 0; c < U; ++c) {
            long o = (long)b * U + c;
            float sc = babsr_score(l[o], u[o], mask[o], weight, o);
            if (sc < 0.0f) continue;
            int rank = 0;
            for (int c2 = 0; c2 < U; ++c2) {
                if (layer_of[c2] != layer_of[c] || c2 == c) continue;
                long o2 = (long)b * U + c2;
                float s2 = babsr_score(l[o2], u[o2], mask[o2], weight, o2);
                if (s2 > sc || (s2 == sc && c2 < c)) ++rank;
            }
            if (rank < k) tgt_ids[n++] = c;
        }
        tgt_off[b + 1] = n;
    }
    return n;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1 (coordinate ascent over several constraints), repeated for     */
/* `sweeps` passes.  Minimises a.x + c over the box subject to G x + h <= 0   */
/* through the dual  max_{beta>=0} (a + beta^T G).xhat - |a + beta^T G|.eps   */
/*                                   + c + beta^T h          (Eq. 3/4).       */
/* For row k with the other multipliers fixed (Theorem 1):                    */
/*   a' = a + sum_{p != k} beta_p G_p                                         */
/*   q_j = -a'_j / G_kj  (G_kj != 0),  w_j = |G_kj| eps_j, sorted by q        */
/*   s_0 = G_k.xhat + h_k + sum w ;  s_i = s_{i-1} - 2 w_(i)                  */
/*   i* = min{ i in 0..n' : s_i <= 0 },  beta_k = max(q_(i*), 0), q_(0)=-inf  */
/* Returns the dual value after the last update; beta (R) is returned too.    */
/* scale (optional) = (|a| + sum beta|G_p|).max(|lo|,|hi|) + |c| + sum beta|h| */
/* ------------------------------------------------------------------------- */
typedef struct { double q; double w; int j; } bp_t;
static int bp_cmp(const void* A, const void* B) {
    const bp_t* x = (const bp_t*)A; const bp_t* y = (const bp_t*)B;
    if (x->q < y->q) return -1;
    if (x->q > y->q) return 1;
    return (x->j < y->j) ? -1 : (x->j > y->j);
}

double orc_complete_clip(int n, const double* a, double c, int R, const double* G,
                         const double* h, const double* lo, const double* hi,
                         int sweeps, double* beta, double* scale) {
    double* xh = (double*)malloc(sizeof(double) * n);
    double* ep = (double*)malloc(sizeof(double) * n);
    double* ap = (double*)malloc(sizeof(double) * n);
    bp_t* bp = (bp_t*)malloc(sizeof(bp_t) * (n > 0 ? n : 1));
    for (int j = 0; j < n; ++j) { xh[j] = 0.5 * (lo[j] + hi[j]); ep[j] = 0.5 * (hi[j] - lo[j]); }
    for (int k = 0; k < R; ++k) beta[k] = 0.0;
    for (int sw = 0; sw < sweeps; ++sw) {
        for (int k = 0; k < R; ++k) {
            const double* gk = G + (long)k * n;
            /* a' = a + sum_{p != k} beta_p G_p */
            for (int j = 0; j < n; ++j) {
                double v = a[j];
                for (int p = 0; p < R; ++p)
                    if (p != k) v += beta[p] * G[(long)p * n + j];
                ap[j] = v;
            }
            int nb = 0;
            double gx = h[k], W = 0.0;
            for (int j = 0; j < n; ++j) {
                gx += gk[j] * xh[j];
                if (gk[j] != 0.0) {
                    bp[nb].q = -ap[j] / gk[j];
                    bp[nb].w = fabs(gk[j]) * ep[j];
                    bp[nb].j = j;
                    W += bp[nb].w;
                    ++nb;
                }
            }
            qsort(bp, nb, sizeof(bp_t), bp_cmp);
            double s = gx + W;
            double bk = 0.0;           /* i* = 0 -> q_(0) = -inf -> beta 0 */
            if (s > 0.0) {
                int found = 0;
                for (int i = 0; i < nb; ++i) {
                    s -= 2.0 * bp[i].w;
                    if (s <= 0.0) { bk = bp[i].q; found = 1; break; }
                }
                if (!found) bk = 0.0;  /* infeasible row: removed by the pre-check */
            }
            beta[k] = bk > 0.0 ? bk : 0.0;
        }
    }
    /* dual objective at the final beta */
    double val = c, sc = fabs(c);
    for (int k = 0; k < R; ++k) { val += beta[k] * h[k]; sc += beta[k] * fabs(h[k]); }
    for (int j = 0; j < n; ++j) {
        double v = a[j], va = fabs(a[j]);
        for (int p = 0; p < R; ++p) { v += beta[p] * G[(long)p * n + j]; va += beta[p] * fabs(G[(long)p * n + j]); }
        val += v * xh[j] - fabs(v) * ep[j];
        sc += va * fmax(fabs(lo[j]), fabs(hi[j]));
    }
    if (scale) *scale = sc;
    free(xh); free(ep); free(ap); free(bp);
    return val;
}

/* The dual objective D(beta) of Eq. 4 at a given beta (any beta >= 0 gives a */
/* valid lower bound: weak duality).                                          */
double orc_dual_value(int n, const double* a, double c, int R, const double* G,
                      const double* h, const double* lo, const double* hi, const double* beta) {
    double val = c;
    for (int k = 0; k < R; ++k) val += beta[k] * h[k];
    for (int j = 0; j < n; ++j) {
        double v = a[j];
        for (int p = 0; p < R; ++p) v += beta[p] * G[(long)p * n + j];
        double xh = 0.5 * (lo[j] + hi[j]), ep = 0.5 * (hi[j] - lo[j]);
        val += v * xh - fabs(v) * ep;
    }
    return val;
}

/* ------------------------------------------------------------------------- */
/* One BaB round over a batch of subdomains (Algorithm 5 lines 8-11 with the  */
/* cached constraints of Section 3.4):                                        */
/*  a2 rows from splits (cached planes) + extra rows                         */
/*  a3 pre-check on the input box                                             */
/*  a4 relaxed clipping (Algorithm 2, or Algorithm 3 for relaxed = 2 / 3),    */
/*     box rounded outward to FP32                                            */
/*  a5 re-concretisation of every cached plane over the clipped box,          */
/*     intersected with the inherited bounds; split signs enforced (standard */
/*     activation BaB) unless enforce_splits = 0 (the paper's relaxed-clipping */
/*     walk-through keeps the split neuron's clipped bounds as they are)      */
/*  a6 complete clipping (Algorithm 1, `sweeps` passes, orc_complete_clip)  */
/*     of every still-unstable target, both sides                             */
/*  a7 CROWN back-substitution of the spec rows C with the subdomain's bounds */
/*  a8 concretisation over the clipped box; verified iff all f_r > 0         */
/* Infeasible subdomains stop at the step that finds them; they report        */
/* lower = +inf and verified = 1 (pruned, Section 3.2).                       */
/* ------------------------------------------------------------------------- */
typedef struct {
    const net_t* net;
    int U; const int* ids; const double* lA; const double* lc; const double* uA; const double* uc;
    const double* root_l; const double* root_u; const double* pscale; const double* zmag;
    const int* slot_of;   /* global id -> cache slot or -1 */
} cache_t;

static void one_subdomain(const cache_t* cc, int b,
                          const double* lo_in, const double* hi_in,
                          const double* l_in, const double* u_in,
                          const int* split_off, const int* split_ids,
                          const int* row_off, const double* Gx, const double* hx,
                          int m, const double* C, const double* t,
                          const double* alpha, int alpha_mode,
                          const int* tgt_off, const int* tgt_ids,
                          int relaxed, int sweeps, int enforce,
                          double* lower, double* lower_scale, double* lo_c, double* hi_c,
                          double* l_o, double* u_o, double* l_sc, double* u_sc,
                          signed char* mask, unsigned char* infeasible, unsigned char* verified,
                          double* fA, double* fc, double* bw) {
    const net_t* n = cc->net;
    int n0 = n->dims[0], U = cc->U, L = n->L;
    const double* lo = lo_in + (long)b * n0;
    const double* hi = hi_in + (long)b * n0;
    int infeas = 0;

    /* a2: assemble rows g.x + h <= 0 */
    int ns = split_off ? split_off[b + 1] - split_off[b] : 0;
    int ne = row_off ? row_off[b + 1] - row_off[b] : 0;
    int Rmax = ns + ne;
    double* G = (double*)malloc(sizeof(double) * (size_t)(Rmax > 0 ? Rmax : 1) * n0);
    double* h = (double*)malloc(sizeof(double) * (Rmax > 0 ? Rmax : 1));
    int* split_slot = (int*)malloc(sizeof(int) * (ns > 0 ? ns : 1));
    int* split_side = (int*)malloc(sizeof(int) * (ns > 0 ? ns : 1));
    int R = 0;
    for (int s = 0; s < ns; ++s) {
        int code = split_ids[split_off[b] + s];
        int side = code > 0 ? 1 : -1;
        int gid = (code > 0 ? code : -code) - 1;
        int slot = cc->slot_of[gid];
        split_slot[s] = slot; split_side[s] = side;
        if (slot < 0) {
            /* a split on a root-stable neuron: no row; contradiction => infeasible */
            int st = cc->root_l[gid] >= 0.0 ? 1 : -1;
            if (st != side) infeas = 1;
            continue;
        }
        double* g = G + (long)R * n0;
        if (side > 0) {   /* z >= 0  =>  -Abar.x - cbar <= 0 */
            for (int q = 0; q < n0; ++q) g[q] = -cc->uA[(long)slot * n0 + q];
            h[R] = -cc->uc[slot];
        } else {          /* z <= 0  =>  Aund.x + cund <= 0 */
            for (int q = 0; q < n0; ++q) g[q] = cc->lA[(long)slot * n0 + q];
            h[R] = cc->lc[slot];
        }
        ++R;
    }
    for (int e = 0; e < ne; ++e) {
        int r = row_off[b] + e;
        memcpy(G + (long)R * n0, Gx + (long)r * n0, sizeof(double) * n0);
        h[R] = hx[r];
        ++R;
    }

    /* a3: pre-check on the input box; keep the active rows in order */
    int Ra = 0;
    for (int k = 0; k < R; ++k) {
        int f = orc_row_check(n0, G + (long)k * n0, h[k], lo, hi, NULL, NULL, NULL);
        if (f == 1) infeas = 1;
        if (f == 0) {
            if (Ra != k) { memmove(G + (long)Ra * n0, G + (long)k * n0, sizeof(double) * n0); h[Ra] = h[k]; }
            ++Ra;
        }
    }

    /* a4: relaxed clipping on the input box, rounded outward: relaxed = 1 the   */
    /* parallel Algorithm 2; 2 the sequential Algorithm 3 over the active rows in */
    /* their order; 3 Algorithm 3 with the rows in the constraint-importance      */
    /* order (distances from the input box centre).  Complete clipping keeps the  */
    /* active rows in their own order either way.                                 */
    double* clo = lo_c + (long)b * n0;
    double* chi = hi_c + (long)b * n0;
    for (int i = 0; i < n0; ++i) { clo[i] = lo[i]; chi[i] = hi[i]; }
    if (relaxed == 1 && !infeas) {
        for (int k = 0; k < Ra; ++k)
            orc_relaxed_clip_row(n0, G + (long)k * n0, h[k], lo, hi, clo, chi);
    } else if ((relaxed == 2 || relaxed == 3) && !infeas && Ra > 0) {
        int* perm = (int*)malloc(sizeof(int) * Ra);
        double* Gs = (double*)malloc(sizeof(double) * (size_t)Ra * n0);
        double* hs = (double*)malloc(sizeof(double) * Ra);
        if (relaxed == 3) orc_row_order(n0, Ra, G, h, lo, hi, perm);
        else for (int k = 0; k < Ra; ++k) perm[k] = k;
        for (int k = 0; k < Ra; ++k) {
            memcpy(Gs + (long)k * n0, G + (long)perm[k] * n0, sizeof(double) * n0);
            hs[k] = h[perm[k]];
        }
        if (orc_relaxed_clip_sequential(n0, Ra, Gs, hs, lo, hi, clo, chi)) infeas = 1;
        free(perm); free(Gs); free(hs);
    }
    for (int i = 0; i < n0; ++i) {
        clo[i] = rdown32(clo[i]);
        chi[i] = rup32(chi[i]);
        if (clo[i] > chi[i]) infeas = 1;
    }

    /* a5: inherited bounds, then re-concretisation over the clipped box */
    double* lb = l_o + (long)b * U;
    double* ub = u_o + (long)b * U;
    double* ls = l_sc + (long)b * U;
    double* us = u_sc + (long)b * U;
    signed char* mk = mask + (long)b * U;
    for (int c = 0; c < U; ++c) {
        int gid = cc->ids[c];
        lb[c] = l_in ? l_in[(long)b * U + c] : cc->root_l[gid];
        ub[c] = u_in ? u_in[(long)b * U + c] : cc->root_u[gid];
        ls[c] = cc->pscale[gid];
        us[c] = cc->pscale[gid];
    }
    if (!infeas) {
        for (int c = 0; c < U; ++c) {
            double vmin, vmax, dum;
            orc_concretize(n0, cc->lA + (long)c * n0, cc->lc[c], clo, chi, &vmin, &dum);
            orc_concretize(n0, cc->uA + (long)c * n0, cc->uc[c], clo, chi, &dum, &vmax);
            if (vmin > lb[c]) lb[c] = vmin;
            if (vmax < ub[c]) ub[c] = vmax;
        }
    }
    /* state: split sides override, else the margin rule */
    for (int c = 0; c < U; ++c) mk[c] = stab_state(lb[c], ub[c]);
    for (int s = 0; s < ns && enforce; ++s) {
        int slot = split_slot[s];
        if (slot < 0) continue;
        if (split_side[s] > 0) { if (lb[slot] < 0.0) lb[slot] = 0.0; mk[slot] = 1; }
        else                   { if (ub[slot] > 0.0) ub[slot] = 0.0; mk[slot] = -1; }
    }
    if (!infeas) for (int c = 0; c < U; ++c) if (lb[c] > ub[c]) infeas = 1;

    /* a6: complete clipping of the still-unstable targets */
    if (!infeas && sweeps > 0 && Ra > 0) {
        double* beta = (double*)malloc(sizeof(double) * Ra);
        double* an = (double*)malloc(sizeof(double) * n0);
        int nt = tgt_off ? tgt_off[b + 1] - tgt_off[b] : U;
        for (int ti = 0; ti < nt; ++ti) {
            int c = tgt_off ? tgt_ids[tgt_off[b] + ti] : ti;
            if (c < 0 || c >= U || mk[c] != 0) continue;
            double sc;
            /* lower side: min of the lower plane; upper side: -min of the negated upper plane */
            double L1 = orc_complete_clip(n0, cc->lA + (long)c * n0, cc->lc[c], Ra, G, h, clo, chi, sweeps, beta, &sc);
            if (L1 > lb[c]) lb[c] = L1;
            if (sc > ls[c]) ls[c] = sc;
            for (int q = 0; q < n0; ++q) an[q] = -cc->uA[(long)c * n0 + q];
            double L2 = orc_complete_clip(n0, an, -cc->uc[c], Ra, G, h, clo, chi, sweeps, beta, &sc);
            if (-L2 < ub[c]) ub[c] = -L2;
            if (sc > us[c]) us[c] = sc;
        }
        free(beta); free(an);
        for (int c = 0; c < U; ++c) {
            if (mk[c] == 0) mk[c] = stab_state(lb[c], ub[c]);
            if (lb[c] > ub[c]) infeas = 1;
        }
    }

    /* a7/a8: CROWN back-substitution of the spec, concretisation */
    infeasible[b] = (unsigned char)infeas;
    if (infeas) {
        for (int r = 0; r < m; ++r) { lower[(long)b * m + r] = INFINITY; lower_scale[(long)b * m + r] = 0.0; }
        verified[b] = 1;
    } else {
        int H = n->H;
        double* hl = (double*)malloc(sizeof(double) * (H > 0 ? H : 1));
        double* hu = (double*)malloc(sizeof(double) * (H > 0 ? H : 1));
        signed char* hs = (signed char*)malloc(H > 0 ? H : 1);
        for (int g = 0; g < H; ++g) {
            hl[g] = cc->root_l[g]; hu[g] = cc->root_u[g];
            hs[g] = stab_state(hl[g], hu[g]);
        }
        for (int c = 0; c < U; ++c) { int g = cc->ids[c]; hl[g] = lb[c]; hu[g] = ub[c]; hs[g] = mk[c]; }
        int nL = n->dims[L];
        double* Lam = (double*)malloc(sizeof(double) * (size_t)m * nL);
        double* bias = (double*)malloc(sizeof(double) * m);
        double* sc = lower_scale + (long)b * m;
        double* L0 = (double*)malloc(sizeof(double) * (size_t)m * n0);
        double* xm = (double*)malloc(sizeof(double) * n0);
        for (int q = 0; q < n0; ++q) xm[q] = fmax(fabs(clo[q]), fabs(chi[q]));
        for (int r = 0; r < m; ++r) { bias[r] = t[r]; sc[r] = fabs(t[r]); }
        memcpy(Lam, C, sizeof(double) * (size_t)m * nL);
        /* the layer products P^(i) = Lam^(i) W^(i), i = 2..L, for the BaBSR weight */
        double* keep[64] = {0};
        if (bw && m > 0)
            for (int i = 2; i <= L; ++i) keep[i] = (double*)malloc(sizeof(double) * (size_t)m * n->dims[i - 1]);
        backward(n, L, m, Lam, hl, hu, hs, alpha ? alpha + (long)b * m * H : NULL, alpha_mode,
                 L0, bias, sc, cc->zmag, xm, (bw && m > 0) ? keep : NULL);
        /* BaBSR weight (Appendix, neuron selection heuristic): the mean over the spec rows of the
           coefficient of the cached neuron's post-activation in the lower bound, i.e. of column q
           of P^(h+1) for neuron q of hidden layer h */
        if (bw && m > 0) {
            for (int c = 0; c < U; ++c) {
                int g = cc->ids[c], h = 1;
                while (h < L - 1 && g >= n->hoff[h + 1]) ++h;
                int q = g - n->hoff[h], nh = n->dims[h];
                double sum = 0.0;
                for (int r = 0; r < m; ++r) sum += keep[h + 1][(long)r * nh + q];
                bw[(long)b * U + c] = sum / m;
            }
            for (int i = 2; i <= L; ++i) free(keep[i]);
        }
        int ver = 1;
        for (int r = 0; r < m; ++r) {
            double vmin;
            orc_concretize(n0, L0 + (long)r * n0, bias[r], clo, chi, &vmin, NULL);
            for (int q = 0; q < n0; ++q) sc[r] += fabs(L0[(long)r * n0 + q]) * xm[q];
            lower[(long)b * m + r] = vmin;
            if (!(vmin > 0.0)) ver = 0;
            if (fA) memcpy(fA + ((long)b * m + r) * n0, L0 + (long)r * n0, sizeof(double) * n0);
            if (fc) fc[(long)b * m + r] = bias[r];
        }
        verified[b] = (unsigned char)ver;
        free(hl); free(hu); free(hs); free(Lam); free(bias); free(L0); free(xm);
    }
    free(G); free(h); free(split_slot); free(split_side);
}

int orc_bound_batch(int L, const int* dims, const double* W, const double* bvec,
                    int U, const int* ids, const double* lA, const double* lc,
                    const double* uA, const double* uc,
                    const double* root_l, const double* root_u, const double* pscale,
                    int B, const double* lo, const double* hi, const double* l_in, const double* u_in,
                    const int* split_off, const int* split_ids,
                    const int* row_off, const double* G, const double* h,
                    int m, const double* C, const double* t,
                    const double* alpha, int alpha_mode,
                    const int* tgt_off, const int* tgt_ids,
                    int relaxed, int sweeps, int enforce_splits,
                    double* lower, double* lower_scale, double* lo_clip, double* hi_clip,
                    double* l_out, double* u_out, double* l_scale, double* u_scale,
                    signed char* mask, unsigned char* infeasible, unsigned char* verified,
                    double* final_A, double* final_c, double* bab_weight, int nthreads) {
    net_t n;
    if (net_init(&n, L, dims, W, bvec)) return -1;
    cache_t cc;
    cc.net = &n; cc.U = U; cc.ids = ids; cc.lA = lA; cc.lc = lc; cc.uA = uA; cc.uc = uc;
    cc.root_l = root_l; cc.root_u = root_u; cc.pscale = pscale;
    int* slot_of = (int*)malloc(sizeof(int) * (n.H > 0 ? n.H : 1));
    double* zmag = (double*)malloc(sizeof(double) * (n.H > 0 ? n.H : 1));
    for (int g = 0; g < n.H; ++g) { slot_of[g] = -1; zmag[g] = fmax(fabs(root_l[g]), fabs(root_u[g])); }
    for (int c = 0; c < U; ++c) slot_of[ids[c]] = c;
    cc.slot_of = slot_of; cc.zmag = zmag;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int b = 0; b < B; ++b)
        one_subdomain(&cc, b, lo, hi, l_in, u_in, split_off, split_ids, row_off, G, h,
                      m, C, t, alpha, alpha_mode, tgt_off, tgt_ids, relaxed, sweeps, enforce_splits,
                      lower, lower_scale, lo_clip, hi_clip, l_out, u_out, l_scale, u_scale,
                      mask, infeasible, verified, final_A, final_c, bab_weight);
    free(slot_of); free(zmag);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Gradient of the spec bounds with respect to the lower slopes alpha        */
/* (alpha-CROWN, Section 2 / Appendix; optimised with Adam in the paper's     */
/* SDP-FO setting).  For one subdomain with given bounds (l, u, state for     */
/* every hidden neuron) and per-row slopes alpha [m x H], returns f [m] and   */
/* grad_alpha [m x H] = grad_f[r] * d f_r / d alpha_{r,j}, by reverse-mode    */
/* differentiation of the back-substitution with the relaxation choices held  */
/* fixed (the convention "P >= 0 selects the lower relaxation" at P = 0).     */
/* ------------------------------------------------------------------------- */
int orc_alpha_grad(int L, const int* dims, const double* W, const double* bvec,
                   const double* hl, const double* hu, const signed char* hs,
                   const double* lo, const double* hi,
                   int m, const double* C, const double* t, const double* alpha,
                   const double* grad_f, double* f_out, double* grad_alpha,
                   const double* beta, const signed char* bsign, double* grad_beta,
                   const double* zmag, double* scale_out) {
    net_t n;
    if (net_init(&n, L, dims, W, bvec)) return -1;
    int n0 = dims[0], H = n.H;
    /* with scale_out: the magnitude scale of every bound (as orc_bound_batch's lower_scale), with the
       hidden neurons' magnitudes zmag (max(|hl|, |hu|) when NULL) */
    double* sc = NULL;
    double* zm = NULL;
    double* xm = NULL;
    if (scale_out) {
        sc = scale_out;
        for (int r = 0; r < m; ++r) sc[r] = fabs(t[r]);
        zm = (double*)malloc(sizeof(double) * (H > 0 ? H : 1));
        for (int g = 0; g < H; ++g) zm[g] = zmag ? zmag[g] : fmax(fabs(hl[g]), fabs(hu[g]));
        xm = (double*)malloc(sizeof(double) * n0);
        for (int q = 0; q < n0; ++q) xm[q] = fmax(fabs(lo[q]), fabs(hi[q]));
    }
    double** keepP = (double**)calloc(L + 1, sizeof(double*));
    for (int i = 2; i <= L; ++i) keepP[i] = (double*)malloc(sizeof(double) * (size_t)m * dims[i - 1]);
    double* Lam = (double*)malloc(sizeof(double) * (size_t)m * dims[L]);
    double* bias = (double*)malloc(sizeof(double) * m);
    double* L0 = (double*)malloc(sizeof(double) * (size_t)m * n0);
    memcpy(Lam, C, sizeof(double) * (size_t)m * dims[L]);
    for (int r = 0; r < m; ++r) bias[r] = t[r];
    backward_beta(&n, L, m, Lam, hl, hu, hs, alpha, 0, L0, bias, sc, zm, xm, keepP, beta, bsign);
    int wmax = 0;
    for (int i = 0; i <= L; ++i) if (dims[i] > wmax) wmax = dims[i];
    double* gl = (double*)malloc(sizeof(double) * wmax);   /* adjoint of Lam^(i) */
    double* gp = (double*)malloc(sizeof(double) * wmax);   /* adjoint of P^(i+1) */
    for (int r = 0; r < m; ++r) {
        double vmin;
        orc_concretize(n0, L0 + (long)r * n0, bias[r], lo, hi, &vmin, NULL);
        f_out[r] = vmin;
        if (sc)
            for (int q = 0; q < n0; ++q) sc[r] += fabs(L0[(long)r * n0 + q]) * xm[q];
        double gf = grad_f ? grad_f[r] : 1.0;
        for (int g = 0; g < H; ++g) grad_alpha[(long)r * H + g] = 0.0;
        if (grad_beta)
            for (int g = 0; g < H; ++g) grad_beta[(long)r * H + g] = 0.0;
        /* d f / d Lam0_q = xhat_q - sign(Lam0_q) eps_q */
        double* gx = (double*)malloc(sizeof(double) * n0);
        for (int q = 0; q < n0; ++q) {
            double xh = 0.5 * (lo[q] + hi[q]), ep = 0.5 * (hi[q] - lo[q]);
            double v = L0[(long)r * n0 + q];
            gx[q] = gf * (xh - (v > 0.0 ? ep : (v < 0.0 ? -ep : 0.0)));
        }
        /* Lam0 = Lam^(1) W^(1), bias += Lam^(1) b^(1) */
        {
            const double* W1 = Wl(&n, 1); const double* b1 = bl(&n, 1);
            for (int j = 0; j < dims[1]; ++j) {
                double v = gf * b1[j];
                for (int q = 0; q < n0; ++q) v += gx[q] * W1[(long)j * n0 + q];
                gl[j] = v;
            }
        }
        free(gx);
        for (int i = 1; i <= L - 1; ++i) {
            /* Lam^(i) = P^(i+1) * D^(i);  bias += P^(i+1) e^(i) */
            const double* P = keepP[i + 1] + (long)r * dims[i];
            int ho = n.hoff[i];
            for (int j = 0; j < dims[i]; ++j) {
                int g = ho + j;
                double a = alpha[(long)r * H + g];
                double dd, ee;
                relu_relax(P[j], hl[g], hu[g], hs[g], a, &dd, &ee);
                if (hs[g] == 0 && P[j] >= 0.0) grad_alpha[(long)r * H + g] = gl[j] * P[j];
                /* Lam^(i)_j = P_j d_j - bsign_j beta_j: d f / d beta_j = -bsign_j dLam^(i)_j */
                if (grad_beta && bsign && bsign[g]) grad_beta[(long)r * H + g] = -(double)bsign[g] * gl[j];
                gp[j] = gl[j] * dd + gf * ee;
            }
            /* P^(i+1) = Lam^(i+1) W^(i+1), bias += Lam^(i+1) b^(i+1) */
            const double* Wn = Wl(&n, i + 1); const double* bn = bl(&n, i + 1);
            for (int k = 0; k < dims[i + 1]; ++k) {
                double v = gf * bn[k];
                for (int j = 0; j < dims[i]; ++j) v += gp[j] * Wn[(long)k * dims[i] + j];
                gl[k] = v;
            }
        }
    }
    for (int i = 2; i <= L; ++i) free(keepP[i]);
    free(keepP); free(Lam); free(bias); free(L0); free(gl); free(gp); free(zm); free(xm);
    return 0;
}

/* Adam ascent step with clamp to [lo, hi] (Kingma & Ba); beta uses [0, inf).  */
void orc_adam_step_range(long n, double* x, double* m1, double* m2, const double* g, int t, double lr,
                         double b1, double b2, double eps, double lo, double hi) {
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (long i = 0; i < n; ++i) {
        m1[i] = b1 * m1[i] + (1.0 - b1) * g[i];
        m2[i] = b2 * m2[i] + (1.0 - b2) * g[i] * g[i];
        double step = lr * (m1[i] / c1) / (sqrt(m2[i] / c2) + eps);
        x[i] = fmin(fmax(x[i] + step, lo), hi);
    }
}

/* Adam ascent step on alpha with clamp to [0, 1] (Kingma & Ba; the paper's   */
/* SDP-FO setting: lr 0.1 decayed by 0.98 per iteration).  t is 1-based.     */
void orc_adam_step(long n, double* alpha, double* m1, double* m2, const double* g,
                   int t, double lr, double b1, double b2, double eps) {
    orc_adam_step_range(n, alpha, m1, m2, g, t, lr, b1, b2, eps, 0.0, 1.0);
}
