/*
 * SNeCT CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 restatement of what the SNeCT hot path computes
 * (network-constrained Tucker decomposition by SGD, Choi & Sael, arXiv 1711.08095).
 * It exists to check the CUDA library; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline arm may load it.  It shares no code with the CUDA library.
 *
 * Layouts (0-based indices, as opposed to the paper's 1-based ones):
 *   G      J1*J2*J3 doubles, g(p,q,r) at (p*J2 + q)*J3 + r
 *   U[n]   I_n*J_n doubles, row i at U[n] + i*J_n
 *   idx    nnz*3 int32 (i, j, k) per entry, val nnz doubles
 *   edges  m*2 int32 undirected gene pairs, each once, weights y
 *
 * Readings of points the paper leaves open (each used below where it applies):
 *   R1  Alg. 1 line 7 writes Collapse(D, n); the update follows the gradient equation
 *       (Sec. 2.3.2), i.e. the mode-n vector G x_{m != n} u_m, computed directly.
 *   R2  Mini-batches (not in the paper): every gradient of a batch is evaluated at the
 *       batch-start parameters and the contributions are SUMMED, so a batch of one entry is
 *       the per-entry SGD step of Alg. 1 with P = 1.
 *   R3  The core step carries no factor P (one deterministic writer).
 *   R4  Network term: one pass per epoch after the entry pass; each gene row k walks its
 *       neighbours in ascending order, u_k <- u_k - eta*lambda_g*y*(u_k - s_j), where s is
 *       the snapshot of the gene factor taken when the pass starts (Alg. 1 line 10 applied
 *       to both endpoints of every edge, each endpoint updating its own row).
 *   R5  Rows observed zero times in the training entries receive no entry-term update and
 *       no L2 term; the counts |Omega^{n,i}| come from the training entries.
 *   R6  Fold-in (Eq. 9) is solved in closed form with the ridge term lambda*||u||^2 / 2
 *       that the per-entry L2 terms of Sec. 2.3.2 add up to for one row.
 *   R7  Top-k: cosine similarity, descending, ties to the lower row index, a zero-norm row
 *       (or query) scores 0.
 *   R13 The lock-free form of Alg. 1 (Sec. 2.3.3) with one worker: entries and network edges
 *       are visited in one given interleaved order; an entry updates its three rows and the
 *       core at once from the values it read (core step eta * P with P = 1); an edge updates
 *       both endpoints from the values read before either changes.
 *   R14 k-means (Sec. 3.1.1): Lloyd's iterations with squared Euclidean distances from given
 *       initial centroids; ties go to the lower centroid index; a centroid with no rows keeps
 *       its place; stop when an assignment pass changes nothing.  Distances are summed over
 *       the coordinates in order, centroids as sums over the rows in ascending order divided
 *       by the count, all in FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GIDX(p, q, r, J2, J3) (((int64_t)(p) * (J2) + (q)) * (J3) + (r))

/* x~ = sum_{p,q,r} g_pqr a_p b_q c_r  (Eq. 2 written entrywise; Alg. 1 lines 5-6). */
static double predict_one(const int32_t *J, const double *G, const double *a, const double *b,
                          const double *c) {
    double s = 0.0;
    for (int p = 0; p < J[0]; ++p)
        for (int q = 0; q < J[1]; ++q)
            for (int r = 0; r < J[2]; ++r)
                s += G[GIDX(p, q, r, J[1], J[2])] * a[p] * b[q] * c[r];
    return s;
}

void oracle_predict(const int32_t *J, const double *G, const double *U1, const double *U2,
                    const double *U3, const int32_t *idx, int64_t n, double *out) {
    for (int64_t e = 0; e < n; ++e) {
        const int32_t *t = idx + 3 * e;
        out[e] = predict_one(J, G, U1 + (int64_t)t[0] * J[0], U2 + (int64_t)t[1] * J[1],
                             U3 + (int64_t)t[2] * J[2]);
    }
}

/* |Omega^{n,i}|: how many training entries have i as their n-th index (symbol table). */
void oracle_counts(const int32_t *I, const int32_t *idx, int64_t n, int64_t *c1, int64_t *c2,
                   int64_t *c3) {
    int64_t *c[3] = {c1, c2, c3};
    for (int m = 0; m < 3; ++m)
        for (int64_t i = 0; i < I[m]; ++i) c[m][i] = 0;
    for (int64_t e = 0; e < n; ++e)
        for (int m = 0; m < 3; ++m) c[m][idx[3 * e + m]] += 1;
}

/* Objective (Eq. 3 with the L2 term of Sec. 2.3.2, plus lambda_g * f_g of the graph
 * regulariser and f_opt = f + lambda_g f_g):
 *   out[0] = 1/2 sum_Omega (x - x~)^2
 *   out[1] = lambda/2 ||G||^2 + lambda/2 sum_n sum_{i: |Omega^{n,i}|>0} ||u_i^(n)||^2
 *   out[2] = f_g = 1/2 sum_edges y ||u^(2)_k1 - u^(2)_k2||^2   (not yet multiplied by lambda_g)
 *   out[3] = out[0] + out[1] + lambda_g * out[2]
 */
void oracle_loss(const int32_t *I, const int32_t *J, double lambda, double lambda_g, const double *G,
                 const double *U1, const double *U2, const double *U3, const int32_t *idx,
                 const double *val, int64_t n, const int32_t *edges, const double *w, int64_t m,
                 double *out) {
    const double *U[3] = {U1, U2, U3};
    double data = 0.0;
    for (int64_t e = 0; e < n; ++e) {
        const int32_t *t = idx + 3 * e;
        double xt = predict_one(J, G, U1 + (int64_t)t[0] * J[0], U2 + (int64_t)t[1] * J[1],
                                U3 + (int64_t)t[2] * J[2]);
        data += 0.5 * (val[e] - xt) * (val[e] - xt);
    }
    double reg = 0.0;
    int64_t PI = (int64_t)J[0] * J[1] * J[2];
    for (int64_t s = 0; s < PI; ++s) reg += G[s] * G[s];
    for (int md = 0; md < 3; ++md) {
        char *seen = (char *)calloc((size_t)I[md] + 1, 1);
        for (int64_t e = 0; e < n; ++e) seen[idx[3 * e + md]] = 1;
        for (int64_t i = 0; i < I[md]; ++i) {
            if (!seen[i]) continue;
            for (int q = 0; q < J[md]; ++q) reg += U[md][i * J[md] + q] * U[md][i * J[md] + q];
        }
        free(seen);
    }
    reg *= 0.5 * lambda;
    double fg = 0.0;
    for (int64_t t = 0; t < m; ++t) {
        const double *u = U2 + (int64_t)edges[2 * t] * J[1];
        const double *v = U2 + (int64_t)edges[2 * t + 1] * J[1];
        double d2 = 0.0;
        for (int q = 0; q < J[1]; ++q) d2 += (u[q] - v[q]) * (u[q] - v[q]);
        fg += 0.5 * w[t] * d2;
    }
    out[0] = data;
    out[1] = reg;
    out[2] = fg;
    out[3] = data + reg + lambda_g * fg;
}

/* Gradient of the per-entry objective of Sec. 2.3.2 at one entry alpha = (i, j, k) (the
 * gradient equation): with r = x~ - x,
 *   ga = r * (G x2 b x3 c) + lambda/|Omega^{1,i}| a      (length J1)
 *   gb = r * (G x1 a x3 c) + lambda/|Omega^{2,j}| b      (length J2)
 *   gc = r * (G x1 a x2 b) + lambda/|Omega^{3,k}| c      (length J3)
 *   gG = r * (a o b o c)   + lambda/|Omega| G            (J1*J2*J3)
 * Returns r. */
static double entry_grads(const int32_t *J, const double *G, const double *a, const double *b,
                          const double *c, double x, double lam_a, double lam_b, double lam_c,
                          double lam_G, double *ga, double *gb, double *gc, double *gG) {
    double r = predict_one(J, G, a, b, c) - x;
    for (int p = 0; p < J[0]; ++p) {
        double s = 0.0;
        for (int q = 0; q < J[1]; ++q)
            for (int r3 = 0; r3 < J[2]; ++r3) s += G[GIDX(p, q, r3, J[1], J[2])] * b[q] * c[r3];
        ga[p] = r * s + lam_a * a[p];
    }
    for (int q = 0; q < J[1]; ++q) {
        double s = 0.0;
        for (int p = 0; p < J[0]; ++p)
            for (int r3 = 0; r3 < J[2]; ++r3) s += G[GIDX(p, q, r3, J[1], J[2])] * a[p] * c[r3];
        gb[q] = r * s + lam_b * b[q];
    }
    for (int r3 = 0; r3 < J[2]; ++r3) {
        double s = 0.0;
        for (int p = 0; p < J[0]; ++p)
            for (int q = 0; q < J[1]; ++q) s += G[GIDX(p, q, r3, J[1], J[2])] * a[p] * b[q];
        gc[r3] = r * s + lam_c * c[r3];
    }
    for (int p = 0; p < J[0]; ++p)
        for (int q = 0; q < J[1]; ++q)
            for (int r3 = 0; r3 < J[2]; ++r3) {
                int64_t s = GIDX(p, q, r3, J[1], J[2]);
                gG[s] = r * a[p] * b[q] * c[r3] + lam_G * G[s];
            }
    return r;
}

/* One mini-batch step of Alg. 1 lines 4-8 under reading R2: entries [start, start+len) of
 * the visit order.  All gradients use the parameters as they were when the batch started;
 * per row and for the core the contributions are summed in entry order, then
 * u <- u - lr * sum, G <- G - lr * sum.  cnt[n] are the training counts |Omega^{n,i}|,
 * n_omega = |Omega| (number of training entries). */
void oracle_batch_step(const int32_t *I, const int32_t *J, double lambda, double lr, double *G,
                       double *U1, double *U2, double *U3, const int32_t *idx, const double *val,
                       int64_t start, int64_t len, const int64_t *cnt1, const int64_t *cnt2,
                       const int64_t *cnt3, int64_t n_omega) {
    double *U[3] = {U1, U2, U3};
    const int64_t *cnt[3] = {cnt1, cnt2, cnt3};
    int64_t PI = (int64_t)J[0] * J[1] * J[2];
    double *snapG = (double *)malloc(sizeof(double) * PI);
    double *sumG = (double *)calloc(PI, sizeof(double));
    double *gG = (double *)malloc(sizeof(double) * PI);
    memcpy(snapG, G, sizeof(double) * PI);
    /* per mode: the sum of the row gradients and a copy of the batch-start rows */
    double *sumU[3], *snapU[3];
    char *touched[3];
    for (int md = 0; md < 3; ++md) {
        sumU[md] = (double *)calloc((size_t)I[md] * J[md], sizeof(double));
        snapU[md] = (double *)malloc(sizeof(double) * (size_t)I[md] * J[md]);
        memcpy(snapU[md], U[md], sizeof(double) * (size_t)I[md] * J[md]);
        touched[md] = (char *)calloc((size_t)I[md], 1);
    }
    double ga[64], gb[64], gc[64];
    for (int64_t e = start; e < start + len; ++e) {
        const int32_t *t = idx + 3 * e;
        const double *a = snapU[0] + (int64_t)t[0] * J[0];
        const double *b = snapU[1] + (int64_t)t[1] * J[1];
        const double *c = snapU[2] + (int64_t)t[2] * J[2];
        entry_grads(J, snapG, a, b, c, val[e], lambda / (double)cnt[0][t[0]],
                    lambda / (double)cnt[1][t[1]], lambda / (double)cnt[2][t[2]],
                    lambda / (double)n_omega, ga, gb, gc, gG);
        const double *g[3] = {ga, gb, gc};
        for (int md = 0; md < 3; ++md) {
            touched[md][t[md]] = 1;
            double *dst = sumU[md] + (int64_t)t[md] * J[md];
            for (int q = 0; q < J[md]; ++q) dst[q] += g[md][q];
        }
        for (int64_t s = 0; s < PI; ++s) sumG[s] += gG[s];
    }
    for (int md = 0; md < 3; ++md) {
        for (int64_t i = 0; i < I[md]; ++i) {
            if (!touched[md][i]) continue;
            for (int q = 0; q < J[md]; ++q) U[md][i * J[md] + q] -= lr * sumU[md][i * J[md] + q];
        }
        free(sumU[md]);
        free(snapU[md]);
        free(touched[md]);
    }
    for (int64_t s = 0; s < PI; ++s) G[s] -= lr * sumG[s];
    free(snapG);
    free(sumG);
    free(gG);
}

/* The data-term part of the gradient equation (Sec. 2.3.2) summed over the entries
 * [start, start+len) of the visit order, every term at the same parameters (as Alg. 1 lines
 * 5-8 evaluate one entry, without the L2 terms): with r = x~ - x per entry,
 *   gA[i] = sum_{e: i_e = i} r (G x2 b x3 c)     I1 x J1
 *   gB[j] = sum_{e: j_e = j} r (G x1 a x3 c)     I2 x J2
 *   gC[k] = sum_{e: k_e = k} r (G x1 a x2 b)     I3 x J3
 *   gG    = sum_e r a o b o c                    J1 x J2 x J3
 * i.e. the gradient of 1/2 sum_e (x_e - x~_e)^2 over the range.  nA (I1 x I3) and nB
 * (I2 x I3) count the range's entries per (patient, platform) and (gene, platform).  Every
 * output is overwritten; sums run in entry order. */
void oracle_data_grad_sums(const int32_t *I, const int32_t *J, const double *G, const double *U1,
                           const double *U2, const double *U3, const int32_t *idx, const double *val,
                           int64_t start, int64_t len, double *gA, double *gB, double *gC, double *gG,
                           double *nA, double *nB) {
    const double *U[3] = {U1, U2, U3};
    double *out[3] = {gA, gB, gC};
    int64_t PI = (int64_t)J[0] * J[1] * J[2];
    for (int md = 0; md < 3; ++md)
        for (int64_t s = 0; s < (int64_t)I[md] * J[md]; ++s) out[md][s] = 0.0;
    for (int64_t s = 0; s < PI; ++s) gG[s] = 0.0;
    for (int64_t s = 0; s < (int64_t)I[0] * I[2]; ++s) nA[s] = 0.0;
    for (int64_t s = 0; s < (int64_t)I[1] * I[2]; ++s) nB[s] = 0.0;
    double *eG = (double *)malloc(sizeof(double) * PI);
    double ga[64], gb[64], gc[64];
    for (int64_t e = start; e < start + len; ++e) {
        const int32_t *t = idx + 3 * e;
        entry_grads(J, G, U[0] + (int64_t)t[0] * J[0], U[1] + (int64_t)t[1] * J[1],
                    U[2] + (int64_t)t[2] * J[2], val[e], 0.0, 0.0, 0.0, 0.0, ga, gb, gc, eG);
        const double *g[3] = {ga, gb, gc};
        for (int md = 0; md < 3; ++md) {
            double *dst = out[md] + (int64_t)t[md] * J[md];
            for (int q = 0; q < J[md]; ++q) dst[q] += g[md][q];
        }
        for (int64_t s = 0; s < PI; ++s) gG[s] += eG[s];
        nA[(int64_t)t[0] * I[2] + t[2]] += 1.0;
        nB[(int64_t)t[1] * I[2] + t[2]] += 1.0;
    }
    free(eG);
}

/* Network term pass (Alg. 1 line 10, reading R4).  The oracle builds its own sorted
 * adjacency from the undirected edge list. */
void oracle_edge_pass(int32_t I2, int32_t J2, double lambda_g, double lr, double *U2,
                      const int32_t *edges, const double *w, int64_t m) {
    if (m == 0 || lambda_g == 0.0) return;
    /* adjacency lists with both directions, neighbours sorted ascending */
    int64_t *deg = (int64_t *)calloc((size_t)I2 + 1, sizeof(int64_t));
    for (int64_t t = 0; t < m; ++t) {
        deg[edges[2 * t]]++;
        deg[edges[2 * t + 1]]++;
    }
    int64_t *ptr = (int64_t *)calloc((size_t)I2 + 1, sizeof(int64_t));
    for (int64_t k = 0; k < I2; ++k) ptr[k + 1] = ptr[k] + deg[k];
    int32_t *nbr = (int32_t *)malloc(sizeof(int32_t) * 2 * m);
    double *wy = (double *)malloc(sizeof(double) * 2 * m);
    int64_t *fill = (int64_t *)calloc((size_t)I2, sizeof(int64_t));
    for (int64_t t = 0; t < m; ++t) {
        int32_t u = edges[2 * t], v = edges[2 * t + 1];
        nbr[ptr[u] + fill[u]] = v;
        wy[ptr[u] + fill[u]++] = w[t];
        nbr[ptr[v] + fill[v]] = u;
        wy[ptr[v] + fill[v]++] = w[t];
    }
    for (int64_t k = 0; k < I2; ++k) { /* insertion sort of each neighbour list */
        for (int64_t s = ptr[k] + 1; s < ptr[k + 1]; ++s) {
            int32_t nv = nbr[s];
            double nw = wy[s];
            int64_t d = s - 1;
            while (d >= ptr[k] && nbr[d] > nv) {
                nbr[d + 1] = nbr[d];
                wy[d + 1] = wy[d];
                --d;
            }
            nbr[d + 1] = nv;
            wy[d + 1] = nw;
        }
    }
    double *snap = (double *)malloc(sizeof(double) * (size_t)I2 * J2);
    memcpy(snap, U2, sizeof(double) * (size_t)I2 * J2);
    for (int64_t k = 0; k < I2; ++k) {
        double *u = U2 + k * J2;
        for (int64_t s = ptr[k]; s < ptr[k + 1]; ++s) {
            const double *v = snap + (int64_t)nbr[s] * J2;
            double st = lr * lambda_g * wy[s];
            for (int q = 0; q < J2; ++q) u[q] -= st * (u[q] - v[q]);
        }
    }
    free(snap);
    free(fill);
    free(wy);
    free(nbr);
    free(ptr);
    free(deg);
}

/* One epoch (Alg. 1 lines 3-13 under R2-R5): the entries in the given order, cut into
 * consecutive batches of `batch` (the last one ragged), then one network-term pass. */
void oracle_epoch(const int32_t *I, const int32_t *J, double lambda, double lambda_g, double lr,
                  int64_t batch, double *G, double *U1, double *U2, double *U3, const int32_t *idx,
                  const double *val, int64_t n, const int32_t *edges, const double *w, int64_t m) {
    int64_t *cnt[3];
    for (int md = 0; md < 3; ++md) cnt[md] = (int64_t *)malloc(sizeof(int64_t) * ((size_t)I[md] + 1));
    oracle_counts(I, idx, n, cnt[0], cnt[1], cnt[2]);
    if (batch <= 0) batch = 1;
    for (int64_t s = 0; s < n; s += batch) {
        int64_t len = (n - s < batch) ? (n - s) : batch;
        oracle_batch_step(I, J, lambda, lr, G, U1, U2, U3, idx, val, s, len, cnt[0], cnt[1],
                          cnt[2], n);
    }
    oracle_edge_pass(I[1], J[1], lambda_g, lr, U2, edges, w, m);
    for (int md = 0; md < 3; ++md) free(cnt[md]);
}

/* Sequential per-entry SGD epoch: Alg. 1 with one worker (P = 1).  Each entry's gradient is
 * evaluated at the current parameters and applied at once (the same step as a mini-batch of
 * one entry, without copying the factor matrices), then one network-term pass (R4). */
void oracle_sgd_epoch(const int32_t *I, const int32_t *J, double lambda, double lambda_g, double lr,
                      double *G, double *U1, double *U2, double *U3, const int32_t *idx,
                      const double *val, int64_t n, const int32_t *edges, const double *w,
                      int64_t m) {
    int64_t *cnt[3];
    for (int md = 0; md < 3; ++md) cnt[md] = (int64_t *)malloc(sizeof(int64_t) * ((size_t)I[md] + 1));
    oracle_counts(I, idx, n, cnt[0], cnt[1], cnt[2]);
    int64_t PI = (int64_t)J[0] * J[1] * J[2];
    double *gG = (double *)malloc(sizeof(double) * PI);
    double ga[64], gb[64], gc[64];
    for (int64_t e = 0; e < n; ++e) {
        const int32_t *t = idx + 3 * e;
        double *a = U1 + (int64_t)t[0] * J[0];
        double *b = U2 + (int64_t)t[1] * J[1];
        double *c = U3 + (int64_t)t[2] * J[2];
        entry_grads(J, G, a, b, c, val[e], lambda / (double)cnt[0][t[0]],
                    lambda / (double)cnt[1][t[1]], lambda / (double)cnt[2][t[2]],
                    lambda / (double)n, ga, gb, gc, gG);
        for (int q = 0; q < J[0]; ++q) a[q] -= lr * ga[q];
        for (int q = 0; q < J[1]; ++q) b[q] -= lr * gb[q];
        for (int q = 0; q < J[2]; ++q) c[q] -= lr * gc[q];
        for (int64_t s = 0; s < PI; ++s) G[s] -= lr * gG[s];
    }
    oracle_edge_pass(I[1], J[1], lambda_g, lr, U2, edges, w, m);
    free(gG);
    for (int md = 0; md < 3; ++md) free(cnt[md]);
}

/* In-place Cholesky factorisation of the SPD matrix A (n x n, row-major) into its lower
 * factor L (A = L L^T), then solves A x = b.  Returns 0, or -1 if A is not positive definite. */
static int cholesky_solve(int n, double *A, double *b) {
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
        if (!(d > 0.0)) return -1;
        d = sqrt(d);
        A[j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = s / d;
        }
    }
    for (int i = 0; i < n; ++i) { /* L y = b */
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= A[i * n + k] * b[k];
        b[i] = s / A[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) { /* L^T x = y */
        double s = b[i];
        for (int k = i + 1; k < n; ++k) s -= A[k * n + i] * b[k];
        b[i] = s / A[i * n + i];
    }
    return 0;
}

/* Fold-in of a new patient (Eq. 9 under R6): with w_jk = G x2 b_j x3 c_k (length J1),
 * u = (sum w w^T + ridge I)^{-1} sum x w over the query's observed (j, k) cells.
 * Returns 0, or -1 if the normal matrix is not positive definite. */
int oracle_foldin(const int32_t *J, const double *G, const double *U2, const double *U3,
                  const int32_t *jk, const double *x, int64_t n, double ridge, double *u_out) {
    int J1 = J[0];
    double *M = (double *)calloc((size_t)J1 * J1, sizeof(double));
    double *rhs = (double *)calloc((size_t)J1, sizeof(double));
    double *wv = (double *)malloc(sizeof(double) * J1);
    for (int64_t e = 0; e < n; ++e) {
        const double *b = U2 + (int64_t)jk[2 * e] * J[1];
        const double *c = U3 + (int64_t)jk[2 * e + 1] * J[2];
        for (int p = 0; p < J1; ++p) {
            double s = 0.0;
            for (int q = 0; q < J[1]; ++q)
                for (int r = 0; r < J[2]; ++r) s += G[GIDX(p, q, r, J[1], J[2])] * b[q] * c[r];
            wv[p] = s;
        }
        for (int p = 0; p < J1; ++p) {
            rhs[p] += x[e] * wv[p];
            for (int q = 0; q < J1; ++q) M[p * J1 + q] += wv[p] * wv[q];
        }
    }
    for (int p = 0; p < J1; ++p) M[p * J1 + p] += ridge;
    int rc = cholesky_solve(J1, M, rhs);
    for (int p = 0; p < J1; ++p) u_out[p] = rhs[p];
    free(wv);
    free(rhs);
    free(M);
    return rc;
}

/* Top-k rows of U1 by cosine similarity to u (reading R7), k <= I1. */
void oracle_topk(const double *U1, int64_t I1, int32_t J1, const double *u, int32_t k,
                 int64_t *idx_out, double *score_out) {
    double nu = 0.0;
    for (int p = 0; p < J1; ++p) nu += u[p] * u[p];
    nu = sqrt(nu);
    double *score = (double *)malloc(sizeof(double) * (size_t)I1);
    char *taken = (char *)calloc((size_t)I1, 1);
    for (int64_t i = 0; i < I1; ++i) {
        double d = 0.0, nr = 0.0;
        for (int p = 0; p < J1; ++p) {
            d += U1[i * J1 + p] * u[p];
            nr += U1[i * J1 + p] * U1[i * J1 + p];
        }
        nr = sqrt(nr);
        score[i] = (nr > 0.0 && nu > 0.0) ? d / (nr * nu) : 0.0;
    }
    for (int32_t t = 0; t < k; ++t) { /* selection: largest score, lowest index on ties */
        int64_t best = -1;
        for (int64_t i = 0; i < I1; ++i) {
            if (taken[i]) continue;
            if (best < 0 || score[i] > score[best]) best = i;
        }
        taken[best] = 1;
        idx_out[t] = best;
        score_out[t] = score[best];
    }
    free(taken);
    free(score);
}

/* QR post-pass (Alg. 1, the step after the sweeps): for each mode, U = Q R (thin,
 * Householder), U <- Q, G <- G x_n R.  A mode with J_n > I_n has no J_n orthonormal columns
 * and keeps its factor (reading R12); returns the bit mask of the modes kept. */
int oracle_qr_post(const int32_t *I, const int32_t *J, double *G, double *U1, double *U2,
                   double *U3) {
    double *U[3] = {U1, U2, U3};
    int skipped = 0;
    int64_t PI = (int64_t)J[0] * J[1] * J[2];
    double *Gn = (double *)malloc(sizeof(double) * PI);
    for (int md = 0; md < 3; ++md) {
        if (J[md] > I[md]) {
            skipped |= 1 << md;
            continue;
        }
        int64_t m = I[md];
        int nc = J[md];
        double *A = U[md];
        double *R = (double *)calloc((size_t)nc * nc, sizeof(double));
        double *V = (double *)calloc((size_t)m * nc, sizeof(double)); /* Householder vectors */
        double *W = (double *)malloc(sizeof(double) * (size_t)m * nc);
        memcpy(W, A, sizeof(double) * (size_t)m * nc);
        for (int j = 0; j < nc; ++j) {
            double nrm = 0.0;
            for (int64_t i = j; i < m; ++i) nrm += W[i * nc + j] * W[i * nc + j];
            nrm = sqrt(nrm);
            double alpha = (W[j * nc + j] > 0.0) ? -nrm : nrm;
            double vn = 0.0;
            for (int64_t i = j; i < m; ++i) {
                V[i * nc + j] = W[i * nc + j] - (i == j ? alpha : 0.0);
                vn += V[i * nc + j] * V[i * nc + j];
            }
            if (vn > 0.0) {
                for (int c = j; c < nc; ++c) {
                    double d = 0.0;
                    for (int64_t i = j; i < m; ++i) d += V[i * nc + j] * W[i * nc + c];
                    double f = 2.0 * d / vn;
                    for (int64_t i = j; i < m; ++i) W[i * nc + c] -= f * V[i * nc + j];
                }
            }
            for (int c = j; c < nc; ++c) R[j * nc + c] = W[j * nc + c];
        }
        /* Q = H_0 H_1 ... H_{nc-1} applied to the first nc columns of the identity */
        for (int64_t i = 0; i < m; ++i)
            for (int c = 0; c < nc; ++c) A[i * nc + c] = (i == c) ? 1.0 : 0.0;
        for (int j = nc - 1; j >= 0; --j) {
            double vn = 0.0;
            for (int64_t i = j; i < m; ++i) vn += V[i * nc + j] * V[i * nc + j];
            if (vn == 0.0) continue;
            for (int c = 0; c < nc; ++c) {
                double d = 0.0;
                for (int64_t i = j; i < m; ++i) d += V[i * nc + j] * A[i * nc + c];
                double f = 2.0 * d / vn;
                for (int64_t i = j; i < m; ++i) A[i * nc + c] -= f * V[i * nc + j];
            }
        }
        /* G <- G x_md R: new g at index t along mode md = sum_s R[t][s] g(.. s ..) */
        for (int p = 0; p < J[0]; ++p)
            for (int q = 0; q < J[1]; ++q)
                for (int r = 0; r < J[2]; ++r) {
                    int t = md == 0 ? p : (md == 1 ? q : r);
                    double s = 0.0;
                    for (int z = 0; z < nc; ++z) {
                        int pp = md == 0 ? z : p, qq = md == 1 ? z : q, rr = md == 2 ? z : r;
                        s += R[t * nc + z] * G[GIDX(pp, qq, rr, J[1], J[2])];
                    }
                    Gn[GIDX(p, q, r, J[1], J[2])] = s;
                }
        memcpy(G, Gn, sizeof(double) * PI);
        free(W);
        free(V);
        free(R);
    }
    free(Gn);
    return skipped;
}

/* Alg. 1 lines 3-13 with one worker (P = 1) in a given interleaved order (reading R13):
 * order[t] < n picks entry order[t] of idx/val, order[t] >= n picks edge order[t] - n.
 * Entry: the per-entry gradients of Sec. 2.3.2 at the current values, then
 * u_in <- u_in - lr g_n for the three rows and G <- G - lr * P * gG with P = 1.
 * Edge (k1, k2, y): u_k1 <- u_k1 - lr lambda_g y (u_k1 - u_k2) and
 * u_k2 <- u_k2 - lr lambda_g y (u_k2 - u_k1), both from the values before the edge.
 * The counts |Omega^{n,i}| come from all n entries. */
void oracle_hogwild_epoch(const int32_t *I, const int32_t *J, double lambda, double lambda_g,
                          double lr, double *G, double *U1, double *U2, double *U3,
                          const int32_t *idx, const double *val, int64_t n, const int32_t *edges,
                          const double *w, int64_t m, const int64_t *order, int64_t n_items) {
    int64_t *cnt[3];
    for (int md = 0; md < 3; ++md) cnt[md] = (int64_t *)malloc(sizeof(int64_t) * ((size_t)I[md] + 1));
    oracle_counts(I, idx, n, cnt[0], cnt[1], cnt[2]);
    int64_t PI = (int64_t)J[0] * J[1] * J[2];
    double *gG = (double *)malloc(sizeof(double) * PI);
    double ga[64], gb[64], gc[64], d[64];
    for (int64_t t = 0; t < n_items; ++t) {
        int64_t it = order[t];
        if (it < n) {
            const int32_t *e = idx + 3 * it;
            double *a = U1 + (int64_t)e[0] * J[0];
            double *b = U2 + (int64_t)e[1] * J[1];
            double *c = U3 + (int64_t)e[2] * J[2];
            entry_grads(J, G, a, b, c, val[it], lambda / (double)cnt[0][e[0]],
                        lambda / (double)cnt[1][e[1]], lambda / (double)cnt[2][e[2]],
                        lambda / (double)n, ga, gb, gc, gG);
            for (int q = 0; q < J[0]; ++q) a[q] -= lr * ga[q];
            for (int q = 0; q < J[1]; ++q) b[q] -= lr * gb[q];
            for (int q = 0; q < J[2]; ++q) c[q] -= lr * gc[q];
            for (int64_t s = 0; s < PI; ++s) G[s] -= lr * gG[s];
        } else {
            int64_t ed = it - n;
            double *u = U2 + (int64_t)edges[2 * ed] * J[1];
            double *v = U2 + (int64_t)edges[2 * ed + 1] * J[1];
            double st = lr * lambda_g * w[ed];
            for (int q = 0; q < J[1]; ++q) d[q] = u[q] - v[q];
            for (int q = 0; q < J[1]; ++q) {
                u[q] -= st * d[q];
                v[q] += st * d[q];
            }
        }
    }
    free(gG);
    for (int md = 0; md < 3; ++md) free(cnt[md]);
}

/* Personalised subtype matrix of one patient profile u (Sec. 3.3): S = G x1 u (J2 x J3),
 * S[q][r] = sum_p g_pqr u_p.  row_norm[q] = ||S[q][:]|| is the weight of gene-mode subtype q
 * for the patient; platform_norm[k] = || (S x3 U3)[:][k] ||, (S x3 U3)[q][k] =
 * sum_r S[q][r] U3[k][r], is the weight of platform k (I3 platforms). */
void oracle_subtype(const int32_t *J, int32_t I3, const double *G, const double *U3, const double *u,
                    double *S, double *row_norm, double *platform_norm) {
    for (int q = 0; q < J[1]; ++q)
        for (int r = 0; r < J[2]; ++r) {
            double acc = 0.0;
            for (int p = 0; p < J[0]; ++p) acc += G[GIDX(p, q, r, J[1], J[2])] * u[p];
            S[q * J[2] + r] = acc;
        }
    for (int q = 0; q < J[1]; ++q) {
        double acc = 0.0;
        for (int r = 0; r < J[2]; ++r) acc += S[q * J[2] + r] * S[q * J[2] + r];
        row_norm[q] = sqrt(acc);
    }
    for (int k = 0; k < I3; ++k) {
        double acc = 0.0;
        for (int q = 0; q < J[1]; ++q) {
            double t = 0.0;
            for (int r = 0; r < J[2]; ++r) t += S[q * J[2] + r] * U3[(int64_t)k * J[2] + r];
            acc += t * t;
        }
        platform_norm[k] = sqrt(acc);
    }
}

/* k-means of the n rows of X (n x d) into k clusters (Sec. 3.1.1 on the patient profiles,
 * reading R14), from the initial centroids cent (k x d, overwritten with the final ones).
 * Each pass assigns every row to its nearest centroid; if no assignment changed, it stops;
 * otherwise every centroid with rows moves to their mean.  At most max_iter passes.  assign
 * (n) gets the last pass's clusters, *inertia the summed squared distance of every row to its
 * assigned centroid among the final ones.  Returns the number of centroid updates made. */
int oracle_kmeans(const double *X, int64_t n, int32_t d, int32_t k, double *cent, int32_t max_iter,
                  int32_t *assign, double *inertia) {
    double *sum = (double *)malloc(sizeof(double) * (size_t)k * d);
    int64_t *cntk = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    int updates = 0;
    for (int64_t i = 0; i < n; ++i) assign[i] = -1;
    for (int it = 0; it < max_iter; ++it) {
        int64_t changed = 0;
        for (int64_t i = 0; i < n; ++i) {
            int best = 0;
            double bd = 0.0;
            for (int c = 0; c < k; ++c) {
                double dist = 0.0;
                for (int p = 0; p < d; ++p) {
                    double t = X[i * d + p] - cent[(int64_t)c * d + p];
                    dist = dist + t * t;
                }
                if (c == 0 || dist < bd) {
                    bd = dist;
                    best = c;
                }
            }
            if (assign[i] != best) ++changed;
            assign[i] = best;
        }
        if (changed == 0) break;
        for (int c = 0; c < k; ++c) {
            cntk[c] = 0;
            for (int p = 0; p < d; ++p) sum[(int64_t)c * d + p] = 0.0;
        }
        for (int64_t i = 0; i < n; ++i) {
            cntk[assign[i]] += 1;
            for (int p = 0; p < d; ++p) sum[(int64_t)assign[i] * d + p] += X[i * d + p];
        }
        for (int c = 0; c < k; ++c)
            if (cntk[c] > 0)
                for (int p = 0; p < d; ++p) cent[(int64_t)c * d + p] = sum[(int64_t)c * d + p] / (double)cntk[c];
        ++updates;
    }
    double tot = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double dist = 0.0;
        for (int p = 0; p < d; ++p) {
            double t = X[i * d + p] - cent[(int64_t)assign[i] * d + p];
            dist = dist + t * t;
        }
        tot += dist;
    }
    *inertia = tot;
    free(sum);
    free(cntk);
    return updates;
}
