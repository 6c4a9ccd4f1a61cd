/*
 * dode_oracle.c -- plain, slow, FP64 reference of the per-day DODE / SPGD path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product links, loads or calls this
 * file: only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header or table with the CUDA library.
 *
 * Every function follows one passage of Ma & Qian, "Estimating multi-year 24/7
 * origin-destination demand using high-granular multi-source traffic data"
 * (arXiv 1901.09266).  Equations are named by their labels in the paper's
 * source: Eq. (cost) is the path travel time by link composition (Sec. 2.4),
 * Eq. (dar) the DAR ratio (Sec. 2.3), Eq. (logit) / (rt) / (flow) the route
 * choice (Sec. 2.6), Eq. (assign) the assignment matrix and Eq. (opt) / (nnls)
 * the NNLS problem (Sec. 2.7 and 3), Algorithm 1 the SPGD method (Sec. 3.3).
 *
 * Readings of points the paper leaves open (all listed in the design notes):
 *  - time is counted in integer ticks; tps ticks per second, ipt ticks per
 *    interval (16 and 4800 for 5-minute intervals);
 *  - link travel time is taken at the link entry interval (Sec. 2.4, the
 *    omega_1 = t^2 - (t^1 + c_1(t^1)) relation) and quantised once, in FP32,
 *    to ticks: c = rint(fl32(fl32(len * 3600 tps) / v)), at least 1 tick;
 *  - a link is observed at its tail (entry), intervals are half open
 *    [t^h, t^{h+1}), mass arriving at or after the end of the day is dropped
 *    (Sec. 2.7, per-day decomposition);
 *  - FIFO (Sec. 2.2) is enforced by a running maximum over departures;
 *  - the route time of departure interval h1 is the leading vehicle's
 *    (departing at t^{h1}) time to the end of the route, in minutes;
 *  - Adagrad (Duchi et al.) with G_0 = 0, q_0 = 0 (unless given), no decay;
 *    g = B^T (B q - x) without the factor 2, exactly as Algorithm 1 prints it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_BAD_SPEED -4
#define OR_ERR_TICK_OVERFLOW -5
#define OR_ERR_OOM -6

/* ------------------------------------------------------------------------ */
/* Network + routes (caller-owned arrays, copied)                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t N;          /* intervals per day */
    int32_t ipt;        /* ticks per interval */
    int32_t tps;        /* ticks per second */
    int32_t A;          /* links */
    float *len_mi;      /* [A] */
    int32_t P;          /* routes */
    int32_t K;          /* OD pairs */
    int32_t *rptr;      /* [P+1] */
    int32_t *rlinks;    /* [rptr[P]] */
    int32_t *rod;       /* [P] */
    int32_t O;          /* observed links */
    int32_t *obs_col;   /* [A]: column of link a in the observation order, -1 if unobserved */
} or_net;

/* One DAR entry rho_{rs}^{ka}(h1, h2) of route k at its j-th link (Eq. (dar)). */
typedef struct {
    int32_t k, j, h1, h2;
    double rho;
} or_dar_entry;

/* One day's model: everything the speeds determine. */
typedef struct {
    const or_net *net;
    int32_t Nh;           /* time horizon in intervals: N, or 2N when the next day is
                             coupled (trips past midnight run on its speeds and land
                             in its first intervals, rows N .. 2N-1 here) */
    int32_t *ticks;       /* [Nh][A] link travel time in ticks, by entry interval */
    int64_t *T;           /* [(rptr[k]+k+j)][N+1] trajectory times, j = 0..beta_k */
    int64_t n_repairs;    /* FIFO repairs applied */
    or_dar_entry *dar;    /* DAR entries */
    int64_t n_dar;
    double *C;            /* [N][P] route time of departure interval h1, minutes */
    double *Cc;           /* [N][P] travel times the route choice uses: this day's C,
                             or a traffic pattern's mean (Eq. (logit)) */
    double theta;
    double *p;            /* [N][P] route choice portion */
    /* assignment matrix B (Eq. (assign)) in COO, observed rows only */
    int64_t nnz;
    int32_t *b_row;       /* h2 * O + o, h2 < Nh */
    int32_t *b_col;       /* h1 * K + od */
    double *b_val;
} or_day;

or_net *or_net_create(int32_t N, int32_t interval_s, int32_t tps, int32_t A, const float *len_mi,
                      int32_t P, int32_t K, const int32_t *rptr, const int32_t *rlinks,
                      const int32_t *rod, int32_t O, const int32_t *obs_links) {
    if (N <= 0 || interval_s <= 0 || tps <= 0 || A <= 0 || P <= 0 || K <= 0 || O < 0) return NULL;
    or_net *n = (or_net *)calloc(1, sizeof(or_net));
    n->N = N;
    n->ipt = interval_s * tps;
    n->tps = tps;
    n->A = A;
    n->P = P;
    n->K = K;
    n->O = O;
    n->len_mi = (float *)malloc(sizeof(float) * A);
    memcpy(n->len_mi, len_mi, sizeof(float) * A);
    n->rptr = (int32_t *)malloc(sizeof(int32_t) * (P + 1));
    memcpy(n->rptr, rptr, sizeof(int32_t) * (P + 1));
    n->rlinks = (int32_t *)malloc(sizeof(int32_t) * (rptr[P] > 0 ? rptr[P] : 1));
    memcpy(n->rlinks, rlinks, sizeof(int32_t) * rptr[P]);
    n->rod = (int32_t *)malloc(sizeof(int32_t) * P);
    memcpy(n->rod, rod, sizeof(int32_t) * P);
    n->obs_col = (int32_t *)malloc(sizeof(int32_t) * A);
    for (int32_t a = 0; a < A; ++a) n->obs_col[a] = -1;
    for (int32_t o = 0; o < O; ++o) n->obs_col[obs_links[o]] = o;
    return n;
}

void or_net_destroy(or_net *n) {
    if (!n) return;
    free(n->len_mi); free(n->rptr); free(n->rlinks); free(n->rod); free(n->obs_col);
    free(n);
}

/* ------------------------------------------------------------------------ */
/* Step 1 -- link travel times from probe speeds (Sec. 2.4, last paragraph): */
/* the travel time of link a entered in interval h, in integer ticks.       */
/* The quantisation is done in IEEE FP32 (multiply, divide, round to        */
/* nearest even) so that any implementation reproduces the same integers.  */
/* ------------------------------------------------------------------------ */
int or_ticks(const or_net *n, const float *speed_mph /* [N][A] */, int32_t *ticks /* [N][A] */) {
    const float scale = (float)(n->tps * 3600);
    for (int32_t h = 0; h < n->N; ++h) {
        for (int32_t a = 0; a < n->A; ++a) {
            float v = speed_mph[(size_t)h * n->A + a];
            if (!(v > 0.0f) || !isfinite(v)) return OR_ERR_BAD_SPEED;
            volatile float num = n->len_mi[a] * scale;  /* fl32(len * 3600 tps) */
            volatile float t = num / v;                  /* fl32(num / v) */
            if (!(t <= 16777216.0f)) return OR_ERR_TICK_OVERFLOW;
            float r = nearbyintf(t);                      /* round half to even */
            int32_t c = (int32_t)r;
            ticks[(size_t)h * n->A + a] = c < 1 ? 1 : c;
        }
    }
    return OR_OK;
}

/* c_a(t): travel time of link a for a vehicle entering it at tick t; the    */
/* table covers Nh intervals and its last row holds for later entries.      */
static int64_t link_time(const or_net *n, const int32_t *ticks, int32_t Nh, int32_t a, int64_t t) {
    int64_t h = t / n->ipt;
    if (h > Nh - 1) h = Nh - 1;
    return ticks[h * n->A + a];
}

static size_t traj_index(const or_net *n, int32_t k, int32_t j, int32_t b) {
    return ((size_t)(n->rptr[k] + k + j)) * (size_t)(n->N + 1) + (size_t)b;
}

/* ------------------------------------------------------------------------ */
/* Step 2 -- leading-vehicle trajectories (Example "DAR matrix computation", */
/* Eq. (cost)).  T_{k,0}(b) = t^b is the departure at interval boundary b;   */
/* T_{k,j+1}(b) = T_{k,j}(b) + c_{a_{k,j}}(T_{k,j}(b)).  FIFO (Sec. 2.2) is   */
/* enforced per link, in increasing b, by T_{k,j}(b) >= T_{k,j}(b-1).        */
/* ------------------------------------------------------------------------ */
void or_trajectories(const or_net *n, const int32_t *ticks, int32_t Nh, int64_t *T, int64_t *n_repairs) {
    int64_t rep = 0;
    for (int32_t k = 0; k < n->P; ++k) {
        int32_t beta = n->rptr[k + 1] - n->rptr[k];
        for (int32_t b = 0; b <= n->N; ++b) {
            T[traj_index(n, k, 0, b)] = (int64_t)n->ipt * b;
            for (int32_t j = 0; j < beta; ++j) {
                int32_t a = n->rlinks[n->rptr[k] + j];
                int64_t t = T[traj_index(n, k, j, b)];
                int64_t nxt = t + link_time(n, ticks, Nh, a, t);
                if (b > 0) {
                    int64_t prev = T[traj_index(n, k, j + 1, b - 1)];
                    if (nxt < prev) { nxt = prev; ++rep; }
                }
                T[traj_index(n, k, j + 1, b)] = nxt;
            }
        }
    }
    *n_repairs = rep;
}

/* ------------------------------------------------------------------------ */
/* Step 3 -- DAR (Eq. (dar)): flow of route k departing in H_{h1} reaches    */
/* the tail of its j-th link spread evenly (Eq. (unif)) over the window     */
/* [T_{k,j}(h1), T_{k,j}(h1+1)); rho(h1,h2) is the share of that window in   */
/* H_{h2}.  A zero-length window puts all mass in the interval containing   */
/* it.  Shares at h2 >= Nh are dropped: after midnight (Nh = N), or past    */
/* the end of the coupled next day (Nh = 2N).                               */
/* ------------------------------------------------------------------------ */
static int64_t dar_emit(const or_net *n, int32_t Nh, const int64_t *T, or_dar_entry *out) {
    int64_t m = 0;
    const int64_t ipt = n->ipt;
    for (int32_t k = 0; k < n->P; ++k) {
        int32_t beta = n->rptr[k + 1] - n->rptr[k];
        for (int32_t j = 0; j < beta; ++j) {
            for (int32_t h1 = 0; h1 < n->N; ++h1) {
                int64_t lo = T[traj_index(n, k, j, h1)];
                int64_t hi = T[traj_index(n, k, j, h1 + 1)];
                if (hi == lo) {
                    int64_t h2 = lo / ipt;
                    if (h2 < Nh) {
                        if (out) { out[m].k = k; out[m].j = j; out[m].h1 = h1; out[m].h2 = (int32_t)h2; out[m].rho = 1.0; }
                        ++m;
                    }
                    continue;
                }
                for (int64_t h2 = lo / ipt; h2 <= (hi - 1) / ipt && h2 < Nh; ++h2) {
                    int64_t s = lo > ipt * h2 ? lo : ipt * h2;
                    int64_t e = hi < ipt * (h2 + 1) ? hi : ipt * (h2 + 1);
                    if (out) {
                        out[m].k = k; out[m].j = j; out[m].h1 = h1; out[m].h2 = (int32_t)h2;
                        out[m].rho = (double)(e - s) / (double)(hi - lo);
                    }
                    ++m;
                }
            }
        }
    }
    return m;
}

/* ------------------------------------------------------------------------ */
/* Step 4 -- route choice (Eq. (logit), (rt)): logit over the routes of one  */
/* OD pair on the route time of the leading vehicle of interval h1.         */
/* ------------------------------------------------------------------------ */
static void route_choice(const or_net *n, const double *C, double theta, double *p) {
    for (int32_t h = 0; h < n->N; ++h) {
        for (int32_t od = 0; od < n->K; ++od) {
            double mx = -INFINITY, den = 0.0;
            for (int32_t k = 0; k < n->P; ++k)
                if (n->rod[k] == od && -theta * C[(size_t)h * n->P + k] > mx) mx = -theta * C[(size_t)h * n->P + k];
            for (int32_t k = 0; k < n->P; ++k)
                if (n->rod[k] == od) den += exp(-theta * C[(size_t)h * n->P + k] - mx);
            for (int32_t k = 0; k < n->P; ++k)
                if (n->rod[k] == od) p[(size_t)h * n->P + k] = exp(-theta * C[(size_t)h * n->P + k] - mx) / den;
        }
    }
}

/* Assignment matrix entries B[(h2,o),(h1,od)] += delta rho p (Eq. (assign)). */
static void assemble_B(or_day *d) {
    const or_net *n = d->net;
    int64_t nnz = 0;
    for (int64_t e = 0; e < d->n_dar; ++e) {
        const or_dar_entry *x = &d->dar[e];
        int32_t a = n->rlinks[n->rptr[x->k] + x->j];
        if (n->obs_col[a] >= 0) ++nnz;
    }
    free(d->b_row); free(d->b_col); free(d->b_val);
    d->b_row = (int32_t *)malloc(sizeof(int32_t) * (nnz ? nnz : 1));
    d->b_col = (int32_t *)malloc(sizeof(int32_t) * (nnz ? nnz : 1));
    d->b_val = (double *)malloc(sizeof(double) * (nnz ? nnz : 1));
    int64_t m = 0;
    for (int64_t e = 0; e < d->n_dar; ++e) {
        const or_dar_entry *x = &d->dar[e];
        int32_t a = n->rlinks[n->rptr[x->k] + x->j];
        int32_t o = n->obs_col[a];
        if (o < 0) continue;
        d->b_row[m] = x->h2 * n->O + o;
        d->b_col[m] = x->h1 * n->K + n->rod[x->k];
        d->b_val[m] = x->rho * d->p[(size_t)x->h1 * n->P + x->k];
        ++m;
    }
    d->nnz = nnz;
}

/* Route-choice portions for a dispersion theta (per minute); rebuilds B.   */
void or_day_set_theta(or_day *d, double theta) {
    d->theta = theta;
    route_choice(d->net, d->Cc, theta, d->p);
    assemble_B(d);
}

/* Travel times of the route choice (Eq. (logit) takes the mean travel time */
/* of each path over the days of a traffic pattern): Cc [N][P] minutes, or  */
/* NULL for this day's own route times.  Recomputes p and B.                */
void or_day_set_choice_times(or_day *d, const double *Cc) {
    const or_net *n = d->net;
    memcpy(d->Cc, Cc ? Cc : d->C, sizeof(double) * (size_t)n->N * n->P);
    or_day_set_theta(d, d->theta);
}

/* Build one day's model from its speeds [N][A]; with speed_next (the next  */
/* day's speeds, or NULL) the day is coupled to the next one: the horizon   */
/* covers both days (see or_solve_coupled).  Returns NULL on error.          */
or_day *or_day_build_coupled(const or_net *n, const float *speed_mph, const float *speed_next, double theta,
                             int *err) {
    or_day *d = (or_day *)calloc(1, sizeof(or_day));
    d->net = n;
    d->Nh = speed_next ? 2 * n->N : n->N;
    const size_t NA = (size_t)n->N * n->A;
    d->ticks = (int32_t *)malloc(sizeof(int32_t) * (size_t)d->Nh * n->A);
    int rc = or_ticks(n, speed_mph, d->ticks);
    if (rc == OR_OK && speed_next) rc = or_ticks(n, speed_next, d->ticks + NA);
    if (rc != OR_OK) {
        if (err) *err = rc;
        free(d->ticks); free(d);
        return NULL;
    }
    size_t ntraj = (size_t)(n->rptr[n->P] + n->P) * (size_t)(n->N + 1);
    d->T = (int64_t *)malloc(sizeof(int64_t) * ntraj);
    or_trajectories(n, d->ticks, d->Nh, d->T, &d->n_repairs);
    d->n_dar = dar_emit(n, d->Nh, d->T, NULL);
    d->dar = (or_dar_entry *)malloc(sizeof(or_dar_entry) * (d->n_dar ? d->n_dar : 1));
    dar_emit(n, d->Nh, d->T, d->dar);
    /* route time in minutes (Eq. (cost)): end of route minus departure */
    d->C = (double *)malloc(sizeof(double) * (size_t)n->N * n->P);
    d->Cc = (double *)malloc(sizeof(double) * (size_t)n->N * n->P);
    d->p = (double *)malloc(sizeof(double) * (size_t)n->N * n->P);
    for (int32_t k = 0; k < n->P; ++k) {
        int32_t beta = n->rptr[k + 1] - n->rptr[k];
        for (int32_t h = 0; h < n->N; ++h)
            d->C[(size_t)h * n->P + k] =
                (double)(d->T[traj_index(n, k, beta, h)] - (int64_t)n->ipt * h) / (double)(60 * n->tps);
    }
    memcpy(d->Cc, d->C, sizeof(double) * (size_t)n->N * n->P);
    or_day_set_theta(d, theta);
    if (err) *err = OR_OK;
    return d;
}

or_day *or_day_build(const or_net *n, const float *speed_mph, double theta, int *err) {
    return or_day_build_coupled(n, speed_mph, NULL, theta, err);
}

void or_day_destroy(or_day *d) {
    if (!d) return;
    free(d->ticks); free(d->T); free(d->dar); free(d->C); free(d->Cc); free(d->p);
    free(d->b_row); free(d->b_col); free(d->b_val);
    free(d);
}

/* ---- accessors for tests ------------------------------------------------ */
int64_t or_day_n_dar(const or_day *d) { return d->n_dar; }
int64_t or_day_nnz(const or_day *d) { return d->nnz; }
int64_t or_day_repairs(const or_day *d) { return d->n_repairs; }
void or_day_get_ticks(const or_day *d, int32_t *out) {
    memcpy(out, d->ticks, sizeof(int32_t) * (size_t)d->net->N * d->net->A);
}
void or_day_get_traj(const or_day *d, int64_t *out) {
    const or_net *n = d->net;
    memcpy(out, d->T, sizeof(int64_t) * (size_t)(n->rptr[n->P] + n->P) * (size_t)(n->N + 1));
}
void or_day_get_dar(const or_day *d, int32_t *kjh /* [n][4] */, double *rho) {
    for (int64_t e = 0; e < d->n_dar; ++e) {
        kjh[4 * e + 0] = d->dar[e].k; kjh[4 * e + 1] = d->dar[e].j;
        kjh[4 * e + 2] = d->dar[e].h1; kjh[4 * e + 3] = d->dar[e].h2;
        rho[e] = d->dar[e].rho;
    }
}
void or_day_get_route_choice(const or_day *d, double *C, double *p) {
    size_t m = (size_t)d->net->N * d->net->P;
    if (C) memcpy(C, d->C, sizeof(double) * m);
    if (p) memcpy(p, d->p, sizeof(double) * m);
}
void or_day_get_B(const or_day *d, int32_t *row, int32_t *col, double *val) {
    memcpy(row, d->b_row, sizeof(int32_t) * d->nnz);
    memcpy(col, d->b_col, sizeof(int32_t) * d->nnz);
    memcpy(val, d->b_val, sizeof(double) * d->nnz);
}

/* ------------------------------------------------------------------------ */
/* Step 5 -- link flows implied by OD flows (Eq. (reverse) with (flow)):     */
/* xhat = B q, rows (h2, o) in the time-major order of Table "DODE framework */
/* variable vectorization".                                                 */
/* ------------------------------------------------------------------------ */
void or_forward(const or_day *d, const double *q /* [N][K] */, double *xhat /* [Nh][O] */) {
    const or_net *n = d->net;
    memset(xhat, 0, sizeof(double) * (size_t)d->Nh * n->O);
    for (int64_t e = 0; e < d->nnz; ++e) xhat[d->b_row[e]] += d->b_val[e] * q[d->b_col[e]];
}

/* Step 6 -- masked residual r = m (B q - x) and loss sum r^2 (Eq. (nnls)). */
double or_residual(const or_day *d, const double *xhat, const float *counts, const uint8_t *mask,
                   double *r) {
    const or_net *n = d->net;
    double loss = 0.0;
    for (size_t i = 0; i < (size_t)n->N * n->O; ++i) {
        r[i] = mask[i] ? xhat[i] - (double)counts[i] : 0.0;
        loss += r[i] * r[i];
    }
    return loss;
}

/* Step 7 -- g = B^T r (Algorithm 1, gradient line, without the factor 2).   */
void or_adjoint(const or_day *d, const double *r /* [Nh][O] */, double *g /* [N][K] */) {
    const or_net *n = d->net;
    memset(g, 0, sizeof(double) * (size_t)n->N * n->K);
    for (int64_t e = 0; e < d->nnz; ++e) g[d->b_col[e]] += d->b_val[e] * r[d->b_row[e]];
}

/* Step 8 -- Adagrad step and projection onto q >= 0 (Algorithm 1).          */
static void adagrad_project(size_t m, const double *g, double eta, double eps, double *q, double *G) {
    for (size_t i = 0; i < m; ++i) {
        G[i] += g[i] * g[i];
        q[i] -= eta * g[i] / (sqrt(G[i]) + eps);
        if (q[i] < 0.0) q[i] = 0.0;
    }
}

/* SplitMix64 (Steele, Lea, Flood 2014) -- the generator for the row order. */
uint64_t or_splitmix64_next(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output number i (0-based) of the SplitMix64 stream that starts at state s: */
/* every step adds the same constant to the state, so the state i steps on   */
/* is s + i * gamma and one more step yields output i.                        */
uint64_t or_splitmix64_at(uint64_t s, uint64_t i) {
    uint64_t st = s + i * 0x9E3779B97F4A7C15ULL;
    return or_splitmix64_next(&st);
}

typedef struct {
    uint64_t key;
    int32_t row;
} or_keyed_row;

static int or_cmp_keyed(const void *a, const void *b) {
    const or_keyed_row *x = (const or_keyed_row *)a, *y = (const or_keyed_row *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->row > y->row) - (x->row < y->row);
}

/* permutate(range(n)) of Algorithm 1 over the observed rows of one day and  */
/* epoch.  Every row id r draws the key = output number r of SplitMix64      */
/* started at seed ^ (day << 32 | epoch); the rows are put in ascending      */
/* order of (key, row id).  Ordering i.i.d. uniform keys gives a uniformly   */
/* random permutation, and a row's key does not depend on which other rows   */
/* are observed.                                                             */
void or_permute_rows(int32_t *rows, int32_t n_rows, uint64_t seed, int32_t day, int32_t epoch) {
    uint64_t s0 = seed ^ (((uint64_t)(uint32_t)day << 32) | (uint64_t)(uint32_t)epoch);
    if (n_rows <= 1) return;
    or_keyed_row *t = (or_keyed_row *)malloc(sizeof(or_keyed_row) * (size_t)n_rows);
    for (int32_t i = 0; i < n_rows; ++i) {
        t[i].key = or_splitmix64_at(s0, (uint64_t)(uint32_t)rows[i]);
        t[i].row = rows[i];
    }
    qsort(t, (size_t)n_rows, sizeof(or_keyed_row), or_cmp_keyed);
    for (int32_t i = 0; i < n_rows; ++i) rows[i] = t[i].row;
    free(t);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 on one day.  row_chunk == 0: one full-row update per epoch;   */
/* row_chunk = b > 0: each epoch permutes the observed rows and updates on  */
/* consecutive chunks of b rows (last chunk partial).  q, G are in/out.     */
/* loss_trace[e] = masked loss at the start of epoch e (may be NULL).        */
/* Returns the masked loss of the final q.                                  */
/* ------------------------------------------------------------------------ */
double or_solve_day(const or_day *d, const float *counts, const uint8_t *mask, int32_t iters,
                    double eta, double eps, int32_t row_chunk, uint64_t seed, int32_t day,
                    double *q, double *G, double *loss_trace) {
    const or_net *n = d->net;
    size_t rows = (size_t)n->N * n->O, cols = (size_t)n->N * n->K;
    double *xhat = (double *)malloc(sizeof(double) * rows);
    double *r = (double *)malloc(sizeof(double) * rows);
    double *g = (double *)malloc(sizeof(double) * cols);
    int32_t *order = NULL, n_obs_rows = 0;
    uint8_t *sel = NULL;
    if (row_chunk > 0) {
        order = (int32_t *)malloc(sizeof(int32_t) * (rows ? rows : 1));
        sel = (uint8_t *)malloc(rows ? rows : 1);
    }
    for (int32_t e = 0; e < iters; ++e) {
        if (row_chunk <= 0) {
            or_forward(d, q, xhat);
            double loss = or_residual(d, xhat, counts, mask, r);
            if (loss_trace) loss_trace[e] = loss;
            or_adjoint(d, r, g);
            adagrad_project(cols, g, eta, eps, q, G);
            continue;
        }
        if (loss_trace) {
            or_forward(d, q, xhat);
            loss_trace[e] = or_residual(d, xhat, counts, mask, r);
        }
        /* observed rows in ascending order, then permuted for this epoch */
        n_obs_rows = 0;
        for (size_t i = 0; i < rows; ++i)
            if (mask[i]) order[n_obs_rows++] = (int32_t)i;
        or_permute_rows(order, n_obs_rows, seed, day, e);
        for (int32_t s = 0; s < n_obs_rows; s += row_chunk) {
            int32_t t = s + row_chunk < n_obs_rows ? s + row_chunk : n_obs_rows;
            memset(sel, 0, rows);
            for (int32_t i = s; i < t; ++i) sel[order[i]] = 1;
            or_forward(d, q, xhat);
            or_residual(d, xhat, counts, sel, r);
            or_adjoint(d, r, g);
            adagrad_project(cols, g, eta, eps, q, G);
        }
    }
    or_forward(d, q, xhat);
    double loss = or_residual(d, xhat, counts, mask, r);
    free(xhat); free(r); free(g); free(order); free(sel);
    return loss;
}

/* ------------------------------------------------------------------------ */
/* Quality check (Step 6 of the framework, Sec. 4; the case study reports   */
/* the R-square between observed and estimated link flow, Sec. 5):          */
/* R^2 = 1 - SS_res / SS_tot over the observed cells, SS_res the masked     */
/* loss of q, SS_tot the squared deviations of the observed counts from     */
/* their mean.  NaN when SS_tot = 0 (no observed cell, or constant counts). */
/* ------------------------------------------------------------------------ */
double or_r2_day(const or_day *d, const float *counts, const uint8_t *mask, const double *q) {
    const or_net *n = d->net;
    size_t rows = (size_t)n->N * n->O;
    double *xhat = (double *)malloc(sizeof(double) * rows);
    double *r = (double *)malloc(sizeof(double) * rows);
    or_forward(d, q, xhat);
    double ss_res = or_residual(d, xhat, counts, mask, r);
    double sum = 0.0, cnt = 0.0;
    for (size_t i = 0; i < rows; ++i)
        if (mask[i]) {
            sum += counts[i];
            cnt += 1.0;
        }
    double mean = cnt > 0.0 ? sum / cnt : 0.0, ss_tot = 0.0;
    for (size_t i = 0; i < rows; ++i)
        if (mask[i]) ss_tot += ((double)counts[i] - mean) * ((double)counts[i] - mean);
    free(xhat);
    free(r);
    return ss_tot > 0.0 ? 1.0 - ss_res / ss_tot : NAN;
}

/* ------------------------------------------------------------------------ */
/* Differentiable form: L(q, theta) = sum m (B q - x)^2.                     */
/* dL/dq = 2 B^T r;  dL/dtheta through p = logit(-theta C) (Eq. (logit)):    */
/* dp_k/dtheta = p_k (-C_k + sum_{k' in od} p_k' C_k').                      */
/* ------------------------------------------------------------------------ */
double or_loss_grad_day(const or_day *d, const float *counts, const uint8_t *mask, const double *q,
                        double *dq, double *dtheta, double *dtheta_abs) {
    const or_net *n = d->net;
    size_t rows = (size_t)n->N * n->O, cols = (size_t)n->N * n->K;
    double *xhat = (double *)malloc(sizeof(double) * rows);
    double *r = (double *)malloc(sizeof(double) * rows);
    or_forward(d, q, xhat);
    double loss = or_residual(d, xhat, counts, mask, r);
    if (dq) {
        or_adjoint(d, r, dq);
        for (size_t i = 0; i < cols; ++i) dq[i] *= 2.0;
    }
    if (dtheta) {
        /* route-level adjoint gp[h1][k] = sum_{j,h2} rho r[h2][a_kj], observed links */
        double *gp = (double *)calloc((size_t)n->N * n->P, sizeof(double));
        for (int64_t e = 0; e < d->n_dar; ++e) {
            const or_dar_entry *x = &d->dar[e];
            int32_t o = n->obs_col[n->rlinks[n->rptr[x->k] + x->j]];
            if (o < 0) continue;
            gp[(size_t)x->h1 * n->P + x->k] += x->rho * r[(size_t)x->h2 * n->O + o];
        }
        double acc = 0.0, acc_abs = 0.0;
        for (int32_t h = 0; h < n->N; ++h) {
            for (int32_t k = 0; k < n->P; ++k) {
                int32_t od = n->rod[k];
                double mean_c = 0.0;
                for (int32_t k2 = 0; k2 < n->P; ++k2)
                    if (n->rod[k2] == od) mean_c += d->p[(size_t)h * n->P + k2] * d->Cc[(size_t)h * n->P + k2];
                double pk = d->p[(size_t)h * n->P + k];
                double dp = pk * (-d->Cc[(size_t)h * n->P + k] + mean_c);
                const double term = 2.0 * q[(size_t)h * n->K + od] * gp[(size_t)h * n->P + k] * dp;
                acc += term;
                acc_abs += fabs(term);
            }
        }
        *dtheta = acc;
        /* sum of |terms|: the scale against which a rounding error of the
           cancelling sum is measured */
        if (dtheta_abs) *dtheta_abs = acc_abs;
        free(gp);
    }
    free(xhat); free(r);
    return loss;
}

/* Dense B (rows Nh*O, cols N*K) for tiny instances.                         */
void or_day_dense_B(const or_day *d, double *Bd) {
    const or_net *n = d->net;
    size_t cols = (size_t)n->N * n->K;
    memset(Bd, 0, sizeof(double) * (size_t)d->Nh * n->O * cols);
    for (int64_t e = 0; e < d->nnz; ++e) Bd[(size_t)d->b_row[e] * cols + d->b_col[e]] += d->b_val[e];
}

/* ------------------------------------------------------------------------ */
/* Multi-day driver: days are independent problems (Sec. 2.7), solved one   */
/* by one (optionally several at once with OpenMP).  Inputs are [D][...]    */
/* slabs; q_inout / G_inout are FP64 [D][N][K]; loss_out [D].                */
/* Returns 0, or the first error code met.                                   */
/* ------------------------------------------------------------------------ */
int or_solve_days(const or_net *n, int32_t D, const int32_t *day_ids, const float *speeds,
                  const float *counts, const uint8_t *mask, double theta, const double *choice_times,
                  int32_t iters, double eta, double eps, int32_t row_chunk, uint64_t seed, int32_t n_threads,
                  double *q_inout, double *G_inout, double *loss_out) {
    int status = OR_OK;
    size_t sA = (size_t)n->N * n->A, sO = (size_t)n->N * n->O, sK = (size_t)n->N * n->K;
    (void)n_threads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
#endif
    for (int32_t i = 0; i < D; ++i) {
        int err = OR_OK;
        or_day *d = or_day_build(n, speeds + sA * i, theta, &err);
        if (!d) {
#ifdef _OPENMP
#pragma omp critical
#endif
            { if (status == OR_OK) status = err; }
            continue;
        }
        if (choice_times) or_day_set_choice_times(d, choice_times + (size_t)n->N * n->P * i);
        loss_out[i] = or_solve_day(d, counts + sO * i, mask + sO * i, iters, eta, eps, row_chunk, seed,
                                   day_ids ? day_ids[i] : i, q_inout + sK * i, G_inout + sK * i, NULL);
        or_day_destroy(d);
    }
    return status;
}

/* Forward for many days: xhat [D][N][O] = B_d q_d.                          */
int or_forward_days(const or_net *n, int32_t D, const float *speeds, const double *q, double theta,
                    int32_t n_threads, double *xhat) {
    int status = OR_OK;
    size_t sA = (size_t)n->N * n->A, sO = (size_t)n->N * n->O, sK = (size_t)n->N * n->K;
    (void)n_threads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
#endif
    for (int32_t i = 0; i < D; ++i) {
        int err = OR_OK;
        or_day *d = or_day_build(n, speeds + sA * i, theta, &err);
        if (!d) {
#ifdef _OPENMP
#pragma omp critical
#endif
            { if (status == OR_OK) status = err; }
            continue;
        }
        or_forward(d, q + sK * i, xhat + sO * i);
        or_day_destroy(d);
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Consecutive days solved jointly.  Sec. 2.7 states the problem over the   */
/* whole period as one NNLS and decomposes it into days, at the price of    */
/* the vehicles that depart before midnight and arrive the next day.  Here  */
/* the days stay coupled: day d's model is built with the next day's speeds */
/* (Nh = 2N), so its B has rows [0, N) on day d and rows [N, 2N) on day     */
/* d + 1.  With x_d = B_d q_d over the whole horizon:                        */
/*   xhat_d = x_d[0, N) + x_{d-1}[N, 2N),   r_d = m_d (xhat_d - x_d),          */
/*   loss_d = |r_d|^2,   g_d = B_d^T [r_d ; r_{d+1}]                           */
/* (Algorithm 1's gradient, without the factor 2).  The last day keeps      */
/* Nh = N: its mass after midnight is dropped as in the per-day problem.    */
/* Algorithm 1 runs with full-row updates on all days at once: per epoch    */
/* the forward of every day, then every day's Adagrad step and projection.  */
/* Days [D][N][A] speeds, [D][N][O] counts / mask, q / G FP64 [D][N][K].     */
/* ------------------------------------------------------------------------ */
static or_day **or_build_coupled_days(const or_net *n, int32_t D, const float *speeds, double theta, int *status) {
    const size_t sA = (size_t)n->N * n->A;
    or_day **days = (or_day **)calloc((size_t)D, sizeof(or_day *));
    *status = OR_OK;
    for (int32_t i = 0; i < D; ++i) {
        int err = OR_OK;
        days[i] = or_day_build_coupled(n, speeds + sA * i, i + 1 < D ? speeds + sA * (i + 1) : NULL, theta, &err);
        if (!days[i]) {
            *status = err;
            for (int32_t j = 0; j < i; ++j) or_day_destroy(days[j]);
            free(days);
            return NULL;
        }
    }
    return days;
}

static void or_free_days(or_day **days, int32_t D) {
    for (int32_t i = 0; i < D; ++i) or_day_destroy(days[i]);
    free(days);
}

/* xhat [D][N][O] of the coupled days; xfull [D][2N][O] is scratch.           */
static void or_forward_coupled_days(or_day **days, int32_t D, const double *q, double *xfull, double *xhat) {
    const or_net *n = days[0]->net;
    const size_t sO = (size_t)n->N * n->O, sK = (size_t)n->N * n->K;
    for (int32_t i = 0; i < D; ++i) {
        memset(xfull + 2 * sO * i, 0, sizeof(double) * 2 * sO);
        or_forward(days[i], q + sK * i, xfull + 2 * sO * i);
    }
    for (int32_t i = 0; i < D; ++i)
        for (size_t c = 0; c < sO; ++c)
            xhat[sO * i + c] = xfull[2 * sO * i + c] + (i > 0 ? xfull[2 * sO * (i - 1) + sO + c] : 0.0);
}

int or_forward_coupled(const or_net *n, int32_t D, const float *speeds, const double *q, double theta,
                       double *xhat) {
    int status = OR_OK;
    or_day **days = or_build_coupled_days(n, D, speeds, theta, &status);
    if (!days) return status;
    double *xfull = (double *)malloc(sizeof(double) * 2 * (size_t)n->N * n->O * D);
    or_forward_coupled_days(days, D, q, xfull, xhat);
    free(xfull);
    or_free_days(days, D);
    return OR_OK;
}

/* Residuals r [D][2N][O]: rows [0, N) of day d hold r_d, rows [N, 2N) hold  */
/* r_{d+1} (zero for the last day).  Returns the per-day losses in loss.     */
static void or_residual_coupled(const or_net *n, int32_t D, const double *xhat, const float *counts,
                                const uint8_t *mask, double *r, double *loss) {
    const size_t sO = (size_t)n->N * n->O;
    for (int32_t i = 0; i < D; ++i) {
        double l = 0.0;
        for (size_t c = 0; c < sO; ++c) {
            const double v = mask[sO * i + c] ? xhat[sO * i + c] - (double)counts[sO * i + c] : 0.0;
            r[2 * sO * i + c] = v;
            if (i > 0) r[2 * sO * (i - 1) + sO + c] = v;
            l += v * v;
        }
        loss[i] = l;
    }
    memset(r + 2 * sO * (D - 1) + sO, 0, sizeof(double) * sO);
}

int or_solve_coupled(const or_net *n, int32_t D, const float *speeds, const float *counts, const uint8_t *mask,
                     double theta, int32_t iters, double eta, double eps, double *q_inout, double *G_inout,
                     double *loss_out, double *loss_trace /* [iters][D] or NULL */) {
    int status = OR_OK;
    or_day **days = or_build_coupled_days(n, D, speeds, theta, &status);
    if (!days) return status;
    const size_t sO = (size_t)n->N * n->O, sK = (size_t)n->N * n->K;
    double *xfull = (double *)malloc(sizeof(double) * 2 * sO * D);
    double *xhat = (double *)malloc(sizeof(double) * sO * D);
    double *r = (double *)malloc(sizeof(double) * 2 * sO * D);
    double *g = (double *)malloc(sizeof(double) * sK);
    for (int32_t e = 0; e < iters; ++e) {
        or_forward_coupled_days(days, D, q_inout, xfull, xhat);
        or_residual_coupled(n, D, xhat, counts, mask, r, loss_out);
        if (loss_trace) memcpy(loss_trace + (size_t)e * D, loss_out, sizeof(double) * D);
        for (int32_t i = 0; i < D; ++i) {
            or_adjoint(days[i], r + 2 * sO * i, g);
            adagrad_project(sK, g, eta, eps, q_inout + sK * i, G_inout + sK * i);
        }
    }
    or_forward_coupled_days(days, D, q_inout, xfull, xhat);
    or_residual_coupled(n, D, xhat, counts, mask, r, loss_out);
    free(xfull); free(xhat); free(r); free(g);
    or_free_days(days, D);
    return OR_OK;
}

/* Differentiable form of the coupled days: per-day loss, dL/dq = 2 g_d and  */
/* dL/dtheta split by the day whose route choice it differentiates          */
/* (dp_k/dtheta = p_k (-C_k + sum_{k' in od} p_k' C_k'), Eq. (logit)).         */
int or_loss_grad_coupled(const or_net *n, int32_t D, const float *speeds, const float *counts,
                         const uint8_t *mask, double theta, const double *q, double *loss, double *dq,
                         double *dtheta, double *dtheta_abs /* per day sum of |terms|, or NULL */) {
    int status = OR_OK;
    or_day **days = or_build_coupled_days(n, D, speeds, theta, &status);
    if (!days) return status;
    const size_t sO = (size_t)n->N * n->O, sK = (size_t)n->N * n->K;
    double *xfull = (double *)malloc(sizeof(double) * 2 * sO * D);
    double *xhat = (double *)malloc(sizeof(double) * sO * D);
    double *r = (double *)malloc(sizeof(double) * 2 * sO * D);
    or_forward_coupled_days(days, D, q, xfull, xhat);
    or_residual_coupled(n, D, xhat, counts, mask, r, loss);
    double *gp = (double *)malloc(sizeof(double) * (size_t)n->N * n->P);
    for (int32_t i = 0; i < D; ++i) {
        const or_day *d = days[i];
        const double *ri = r + 2 * sO * i;
        or_adjoint(d, ri, dq + sK * i);
        for (size_t c = 0; c < sK; ++c) dq[sK * i + c] *= 2.0;
        memset(gp, 0, sizeof(double) * (size_t)n->N * n->P);
        for (int64_t e = 0; e < d->n_dar; ++e) {
            const or_dar_entry *x = &d->dar[e];
            int32_t o = n->obs_col[n->rlinks[n->rptr[x->k] + x->j]];
            if (o < 0) continue;
            gp[(size_t)x->h1 * n->P + x->k] += x->rho * ri[(size_t)x->h2 * n->O + o];
        }
        double acc = 0.0, acc_abs = 0.0;
        for (int32_t h = 0; h < n->N; ++h)
            for (int32_t k = 0; k < n->P; ++k) {
                const int32_t od = n->rod[k];
                double mean_c = 0.0;
                for (int32_t k2 = 0; k2 < n->P; ++k2)
                    if (n->rod[k2] == od) mean_c += d->p[(size_t)h * n->P + k2] * d->Cc[(size_t)h * n->P + k2];
                const double pk = d->p[(size_t)h * n->P + k];
                const double term = 2.0 * q[sK * i + (size_t)h * n->K + od] * gp[(size_t)h * n->P + k] * pk *
                                    (-d->Cc[(size_t)h * n->P + k] + mean_c);
                acc += term;
                acc_abs += fabs(term);
            }
        dtheta[i] = acc;
        if (dtheta_abs) dtheta_abs[i] = acc_abs;
    }
    free(gp); free(xfull); free(xhat); free(r);
    or_free_days(days, D);
    return OR_OK;
}

/* Horizon (intervals) and DAR entries of day i of D coupled days (tests).   */
int or_coupled_day_dar(const or_net *n, int32_t D, int32_t i, const float *speeds, int32_t *Nh, int64_t *n_dar,
                       int32_t *kjh /* [n][4] or NULL */, double *rho /* or NULL */) {
    const size_t sA = (size_t)n->N * n->A;
    int err = OR_OK;
    or_day *d = or_day_build_coupled(n, speeds + sA * i, i + 1 < D ? speeds + sA * (i + 1) : NULL, 0.0, &err);
    if (!d) return err;
    *Nh = d->Nh;
    *n_dar = d->n_dar;
    if (kjh && rho) or_day_get_dar(d, kjh, rho);
    or_day_destroy(d);
    return OR_OK;
}
