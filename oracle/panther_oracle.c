/*
 * Panther / Panther++ CPU ORACLE.
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, slow, single-threaded
 * statement of what the GPU path computes. Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the product path never
 * calls it and shares no code, header, table or constant with it.
 *
 * Paper: Zhang, Tang, Ma, Tong, Jing, Li, "Panther: Fast Top-k Similarity
 * Search in Large Networks" (arXiv 1504.02577, KDD 2015).
 *
 * What each function follows:
 *   po_sample_size      Theorem 1 with Lemma 1 ("Sample Size Guarantee", Sec. 3.2)
 *   po_select_prefix    Eq. (3) transition probability t_ij = w_ij / sum_k w_ik
 *   po_alias_row        Eq. (3), realised by an exact integer alias table
 *   po_sample_paths     Algorithm 3 (GenerateRandomPath), Sec. 3.1
 *   po_build_index      the vertex-to-path inverted index P_v (Sec. 3.1, Alg. 3)
 *   po_topk             Algorithm 1 (count each unique co-occurring vertex of
 *                       every path in P_v once), Eq. (4), then top-k
 *   po_theta            Sec. 3.3 feature vector theta(v): the D largest S_RP
 *   po_stream_counts    Eq. (4) and |P_v| from their definitions, path by path,
 *                       with no index (for path sets too large to hold)
 *   po_knn              Sec. 3.3 S_RP++ = 1 / ||theta(v_i) - theta(v_j)||
 *
 * Readings of points the paper leaves open (kept identical on both sides):
 *   - exactly R paths of exactly T+1 vertices (the loop conditions printed in
 *     Algorithm 3 are inverted);
 *   - P_v is a set: a path that visits v twice is listed once;
 *   - the query vertex itself is not a candidate (top-k ranks the OTHER
 *     vertices); theta excludes it too;
 *   - a vertex with no neighbour keeps the walk where it is (the draw for that
 *     step is still consumed, so later steps keep their counters);
 *   - ranking is by integer count desc, then vertex id asc (count/R orders the
 *     same); k-NN ranks by exact squared distance asc, then id asc;
 *   - fewer than k candidates: pad with id -1 (count 0, or distance UINT64_MAX);
 *   - R is rounded up.
 *
 * Random draws: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written
 * here from its published definition. Draw (r, t, attempt) of stream s uses
 *   key = (lo32(seed), hi32(seed)), counter = (lo32(r), hi32(r), (s<<16)|t, attempt)
 * and Uniform[0,S) is Lemire's multiply-shift with rejection (ACM TOMACS
 * 2019): U = x0 | x1<<32, m = U*S (128-bit); reject if low64(m) < 2^64 mod S
 * (then attempt+1), else return high64(m).
 *
 * All-core driver (the po_mt_* functions at the end): the outer loops of the
 * method are independent (paths by id, table rows by vertex, index lists by
 * vertex, queries by id), and the paper's Implementation Notes mention running
 * them in parallel. Each po_mt_* function only cuts one such loop into
 * contiguous ranges and runs the single-threaded code above on every range in
 * its own POSIX thread; it adds no arithmetic of its own, so its output is
 * identical to the single-threaded call (checked by the CPU tests).
 *
 * Parity pins (what holds this file to something other than itself): see the
 * CPU tests. Philox itself has no CPU pin beyond bijectivity and uniformity;
 * its pin is the GPU cross-check against curand's Philox4_32_10.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef unsigned __int128 po_u128;

/* ------------------------------------------------------------- Philox --- */
void po_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The four words of draw (r, t, attempt) on stream s. */
void po_draw(uint64_t seed, uint32_t stream, uint64_t r, uint32_t t, uint32_t attempt, uint32_t out[4]) {
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { (uint32_t)r, (uint32_t)(r >> 32), (stream << 16) | t, attempt };
    po_philox4x32_10(ctr, key, out);
}

/* Lemire: returns 1 and sets *out if U is accepted for range S (S >= 1). */
int po_lemire(uint64_t U, uint64_t S, uint64_t* out) {
    po_u128 m = (po_u128)U * S;
    uint64_t lo = (uint64_t)m;
    if (lo < S) {
        uint64_t thr = (0 - S) % S;            /* (2^64 - S) mod S = 2^64 mod S */
        if (lo < thr) return 0;
    }
    *out = (uint64_t)(m >> 64);
    return 1;
}

/* ------------------------------------------------------ sample size R --- */
/* Theorem 1: |S| = c/eps^2 (d + ln 1/delta); Lemma 1: d = log2 C(T,2) + 1.
 * Returns -1 when the formula is undefined (T < 2 or parameters out of range). */
int64_t po_sample_size(double eps, double delta, double c, int T) {
    if (!(eps > 0 && eps < 1) || !(delta > 0 && delta < 1) || !(c > 0) || T < 2) return -1;
    double pairs = (double)T * (double)(T - 1) / 2.0;         /* C(T, 2) */
    double d = log2(pairs) + 1.0;
    double R = c / (eps * eps) * (d + log(1.0 / delta));
    return (int64_t)ceil(R);
}

/* ------------------------------------------------------------ Eq. (3) --- */
/* Prefix selection: the unique j with sum_{i<j} w_i <= x < sum_{i<=j} w_i,
 * for x drawn uniformly in [0, sum w). Linear scan. */
int64_t po_select_prefix(const uint32_t* w, int64_t d, uint64_t x) {
    uint64_t acc = 0;
    for (int64_t j = 0; j < d; ++j) {
        acc += w[j];
        if (x < acc) return j;
    }
    return -1;
}

/* Integer alias table of one row (Vose): q_j = w_j * d, every column holds
 * capacity S = sum w. Worklists are filled in ascending j; each step takes the
 * LAST small and the LAST large entry; leftovers get thr = S, alias = self.
 * Column c with coin u in [0,S) selects c if u < thr[c], else alias[c]. */
void po_alias_row(const uint32_t* w, int64_t d, uint64_t* thr, int32_t* alias) {
    uint64_t S = 0;
    for (int64_t j = 0; j < d; ++j) S += w[j];
    uint64_t* q = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(d > 0 ? d : 1));
    int64_t* small = (int64_t*)malloc(sizeof(int64_t) * (size_t)(d > 0 ? d : 1));
    int64_t* large = (int64_t*)malloc(sizeof(int64_t) * (size_t)(d > 0 ? d : 1));
    int64_t ns = 0, nl = 0;
    for (int64_t j = 0; j < d; ++j) {
        q[j] = (uint64_t)w[j] * (uint64_t)d;
        if (q[j] < S) small[ns++] = j; else large[nl++] = j;
    }
    while (ns > 0 && nl > 0) {
        int64_t s = small[--ns];
        int64_t l = large[--nl];
        thr[s] = q[s];
        alias[s] = (int32_t)l;
        q[l] -= S - q[s];
        if (q[l] < S) small[ns++] = l; else large[nl++] = l;
    }
    while (nl > 0) { int64_t l = large[--nl]; thr[l] = S; alias[l] = (int32_t)l; }
    while (ns > 0) { int64_t s = small[--ns]; thr[s] = S; alias[s] = (int32_t)s; }
    free(q); free(small); free(large);
}

int64_t po_select_alias(const uint64_t* thr, const int32_t* alias, int64_t d, uint64_t c, uint64_t u) {
    if ((int64_t)c >= d) return -1;
    return u < thr[c] ? (int64_t)c : (int64_t)alias[c];
}

/* Alias tables of every row, in CSR order. */
void po_alias_tables(int64_t n, const int64_t* row_ptr, const uint32_t* w, uint64_t* thr, int32_t* alias) {
    for (int64_t v = 0; v < n; ++v) {
        int64_t s = row_ptr[v], d = row_ptr[v + 1] - s;
        if (d > 0) po_alias_row(w + s, d, thr + s, alias + s);
    }
}

/* ------------------------------------------------------- Algorithm 3 --- */
/* Row sums S_v = sum_j w_vj of rows v0..v1-1 (the denominator of Eq. 3). */
void po_row_sums(int64_t v0, int64_t v1, const int64_t* row_ptr, const uint32_t* w, uint64_t* S) {
    for (int64_t v = v0; v < v1; ++v) {
        uint64_t acc = 0;
        for (int64_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) acc += w[j];
        S[v] = acc;
    }
}

/* Paths r0..r1-1, each T+1 vertices, written row-major to out[(r-r0)*(T+1)+i].
 * mode 0 = prefix selection, 1 = alias selection (thr/alias from
 * po_alias_tables; ignored in prefix mode). rowsum (may be NULL) holds S_v of
 * every row from po_row_sums; without it S_v is summed at every step (the
 * same value). Returns 0, or -1 on bad input. */
int po_sample_paths_rs(int64_t n, const int64_t* row_ptr, const int32_t* col, const uint32_t* w,
                       const uint64_t* thr, const int32_t* alias, const uint64_t* rowsum,
                       uint64_t seed, int64_t r0, int64_t r1, int T, int mode, int32_t* out) {
    if (n < 1 || T < 0 || T > 65535 || (mode != 0 && mode != 1)) return -1;
    int L = T + 1;
    for (int64_t r = r0; r < r1; ++r) {
        int32_t* p = out + (r - r0) * L;
        uint32_t x[4];
        uint64_t v = 0;
        /* start vertex: uniform over V (Alg. 3, "sample current vertex uniformly") */
        for (uint32_t att = 0;; ++att) {
            po_draw(seed, 0, (uint64_t)r, 0, att, x);
            uint64_t U = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
            if (po_lemire(U, (uint64_t)n, &v)) break;
        }
        p[0] = (int32_t)v;
        /* T steps, each to a neighbour with probability t_ij (Eq. 3) */
        for (int t = 1; t <= T; ++t) {
            int64_t s = row_ptr[v], d = row_ptr[v + 1] - s;
            if (d == 0) { p[t] = (int32_t)v; continue; }    /* isolated: stay put */
            uint64_t S = 0;
            if (rowsum) S = rowsum[v];
            else for (int64_t j = 0; j < d; ++j) S += w[s + j];
            int64_t j = -1;
            for (uint32_t att = 0;; ++att) {
                po_draw(seed, 0, (uint64_t)r, (uint32_t)t, att, x);
                uint64_t U0 = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
                if (mode == 0) {
                    uint64_t xr;
                    if (!po_lemire(U0, S, &xr)) continue;
                    j = po_select_prefix(w + s, d, xr);
                    break;
                } else {
                    uint64_t U1 = (uint64_t)x[2] | ((uint64_t)x[3] << 32);
                    uint64_t c, u;
                    int ok0 = po_lemire(U0, (uint64_t)d, &c);
                    int ok1 = po_lemire(U1, S, &u);
                    if (!ok0 || !ok1) continue;
                    j = po_select_alias(thr + s, alias + s, d, c, u);
                    break;
                }
            }
            v = (uint64_t)col[s + j];
            p[t] = (int32_t)v;
        }
    }
    return 0;
}

int po_sample_paths(int64_t n, const int64_t* row_ptr, const int32_t* col, const uint32_t* w,
                    const uint64_t* thr, const int32_t* alias,
                    uint64_t seed, int64_t r0, int64_t r1, int T, int mode, int32_t* out) {
    return po_sample_paths_rs(n, row_ptr, col, w, thr, alias, NULL, seed, r0, r1, T, mode, out);
}

/* --------------------------------------------------- inverted index --- */
static int po_seen_before(const int32_t* p, int i) {
    for (int j = 0; j < i; ++j) if (p[j] == p[i]) return 1;
    return 0;
}

/* off[v] = number of paths containing v, as exclusive prefix (off[n] = nnz).
 * Pass pid = NULL to get off only; then call again with pid sized off[n].
 * P_v lists the ids r of the paths that contain v, ascending, each once. */
int64_t po_build_index(int64_t n, int64_t R, int L, const int32_t* paths, int64_t* off, int32_t* pid) {
    memset(off, 0, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t r = 0; r < R; ++r) {
        const int32_t* p = paths + r * L;
        for (int i = 0; i < L; ++i)
            if (!po_seen_before(p, i)) off[p[i] + 1]++;
    }
    for (int64_t v = 0; v < n; ++v) off[v + 1] += off[v];
    if (pid) {
        int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        memcpy(cur, off, sizeof(int64_t) * (size_t)n);
        for (int64_t r = 0; r < R; ++r) {
            const int32_t* p = paths + r * L;
            for (int i = 0; i < L; ++i)
                if (!po_seen_before(p, i)) pid[cur[p[i]]++] = (int32_t)r;
        }
        free(cur);
    }
    return off[n];
}

/* The same index restricted to the vertices v0 <= v < v1 (every path is
 * still scanned in ascending id): cnt[v - v0] = |P_v| on the first call
 * (pid == NULL); with pid, P_v is written at pid[cur[v - v0]++], cur holding
 * the start of each list. Used by the all-core driver, one vertex range per
 * thread. */
void po_index_range(int64_t R, int L, const int32_t* paths, int64_t v0, int64_t v1, int64_t* cnt_or_cur,
                    int32_t* pid) {
    for (int64_t r = 0; r < R; ++r) {
        const int32_t* p = paths + r * L;
        for (int i = 0; i < L; ++i) {
            int64_t u = p[i];
            if (u < v0 || u >= v1 || po_seen_before(p, i)) continue;
            if (pid) pid[cnt_or_cur[u - v0]++] = (int32_t)r;
            else cnt_or_cur[u - v0]++;
        }
    }
}

/* ------------------------------------------------------- Algorithm 1 --- */
typedef struct { uint32_t cnt; int32_t id; } po_cand;

static int po_cmp_cand(const void* a, const void* b) {
    const po_cand* x = (const po_cand*)a;
    const po_cand* y = (const po_cand*)b;
    if (x->cnt != y->cnt) return x->cnt > y->cnt ? -1 : 1;     /* count desc */
    return (x->id > y->id) - (x->id < y->id);                  /* id asc */
}

/* Counts cnt(v,u) = |{p in P_v : u in p}| for u != v, every unique vertex of
 * a path counted once (Alg. 1), sorted by (count desc, id asc).
 * work_cnt: n zeroed uint32 (left zeroed on return). Returns the number of
 * candidates written to cands (caller sizes it >= min(n, (L-1)*|P_v|)). */
static int64_t po_counts(int64_t n, int L, const int32_t* paths, const int64_t* off, const int32_t* pid,
                         int32_t v, uint32_t* work_cnt, po_cand* cands) {
    int64_t m = 0;
    int64_t cap = (off[v + 1] - off[v]) * (int64_t)(L - 1);
    if (cap > n) cap = n;
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
    for (int64_t e = off[v]; e < off[v + 1]; ++e) {
        const int32_t* p = paths + (int64_t)pid[e] * L;
        for (int i = 0; i < L; ++i) {
            int32_t u = p[i];
            if (u == v || po_seen_before(p, i)) continue;      /* unique u != v */
            if (work_cnt[u] == 0) list[m++] = u;
            work_cnt[u] += 1;                                  /* S_RP(v,u) += 1/R */
        }
    }
    for (int64_t i = 0; i < m; ++i) {
        cands[i].cnt = work_cnt[list[i]];
        cands[i].id = list[i];
        work_cnt[list[i]] = 0;
    }
    free(list);
    qsort(cands, (size_t)m, sizeof(po_cand), po_cmp_cand);
    return m;
}

/* Top-k of query v: ids[k], cnts[k], padded with (-1, 0). Returns #candidates. */
int64_t po_topk(int64_t n, int L, const int32_t* paths, const int64_t* off, const int32_t* pid,
                int32_t v, int k, uint32_t* work_cnt, int32_t* ids, uint32_t* cnts) {
    int64_t cap = (off[v + 1] - off[v]) * (int64_t)(L - 1);
    if (cap > n) cap = n;
    po_cand* c = (po_cand*)malloc(sizeof(po_cand) * (size_t)(cap > 0 ? cap : 1));
    int64_t m = po_counts(n, L, paths, off, pid, v, work_cnt, c);
    for (int i = 0; i < k; ++i) {
        if (i < m) { ids[i] = c[i].id; cnts[i] = c[i].cnt; }
        else { ids[i] = -1; cnts[i] = 0; }
    }
    free(c);
    return m;
}

/* Eq. (4) without an index: paths r0..r1-1 are drawn one at a time, exactly
 * as po_sample_paths_rs draws them, and dropped after use. For every
 * distinct vertex v of a path npaths[v] += 1 (|P_v|, the length of v's list
 * in the inverted index). If v is a query (qpos[v] = i >= 0; -1 for every
 * other vertex), cnt[i*n + u] += 1 for every distinct u != v of the same
 * path: cnt(v, u) as Eq. (4) defines it, the number of paths holding both v
 * and u. Adds to cnt and npaths (the caller zeroes them). Returns 0, or -1
 * on bad input. */
int po_stream_counts(int64_t n, const int64_t* row_ptr, const int32_t* col, const uint32_t* w,
                     const uint64_t* thr, const int32_t* alias, const uint64_t* rowsum,
                     uint64_t seed, int64_t r0, int64_t r1, int T, int mode,
                     const int32_t* qpos, uint64_t* cnt, int64_t* npaths) {
    if (n < 1 || T < 0 || T > 65535 || (mode != 0 && mode != 1) || r1 < r0) return -1;
    int L = T + 1;
    int32_t* p = (int32_t*)malloc(sizeof(int32_t) * (size_t)L);
    if (!p) return -1;
    for (int64_t r = r0; r < r1; ++r) {
        if (po_sample_paths_rs(n, row_ptr, col, w, thr, alias, rowsum, seed, r, r + 1, T, mode, p)) {
            free(p);
            return -1;
        }
        for (int i = 0; i < L; ++i) {
            if (po_seen_before(p, i)) continue;
            npaths[p[i]] += 1;
            int32_t q = qpos[p[i]];
            if (q < 0) continue;
            for (int j = 0; j < L; ++j)
                if (p[j] != p[i] && !po_seen_before(p, j)) cnt[(int64_t)q * n + p[j]] += 1;
        }
    }
    free(p);
    return 0;
}

/* Sec. 3.3: theta(v) = the D largest S_RP(v, u) over u != v, as counts,
 * descending, zero-padded. */
void po_theta(int64_t n, int L, const int32_t* paths, const int64_t* off, const int32_t* pid,
              int32_t v, int D, uint32_t* work_cnt, uint32_t* theta) {
    int64_t cap = (off[v + 1] - off[v]) * (int64_t)(L - 1);
    if (cap > n) cap = n;
    po_cand* c = (po_cand*)malloc(sizeof(po_cand) * (size_t)(cap > 0 ? cap : 1));
    int64_t m = po_counts(n, L, paths, off, pid, v, work_cnt, c);
    for (int d = 0; d < D; ++d) theta[d] = d < m ? c[d].cnt : 0;
    free(c);
}

/* ------------------------------------------------ Panther++ k-NN --- */
typedef struct { uint64_t d2; int32_t id; } po_nb;

static int po_cmp_nb(const void* a, const void* b) {
    const po_nb* x = (const po_nb*)a;
    const po_nb* y = (const po_nb*)b;
    if (x->d2 != y->d2) return x->d2 < y->d2 ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Exact squared Euclidean distance between two count vectors. Returns 0 and
 * sets *out, or -1 if the sum does not fit in 64 bits. */
int po_dist2(const uint32_t* a, const uint32_t* b, int D, uint64_t* out) {
    po_u128 s = 0;
    for (int d = 0; d < D; ++d) {
        int64_t diff = (int64_t)a[d] - (int64_t)b[d];
        s += (po_u128)((po_u128)(diff < 0 ? -diff : diff) * (po_u128)(diff < 0 ? -diff : diff));
    }
    if (s >> 64) return -1;
    *out = (uint64_t)s;
    return 0;
}

/* k nearest u != v by (||theta_v - theta_u||^2 asc, id asc), over all n
 * vectors (theta row-major [n][D]). Ranking by squared distance is the same
 * as ranking by S_RP++ = 1/||.|| descending, and needs no reciprocal.
 * Returns 0, or -1 on overflow. */
int po_knn(int64_t n, int D, const uint32_t* theta, int32_t v, int k, int32_t* ids, uint64_t* d2) {
    po_nb* all = (po_nb*)malloc(sizeof(po_nb) * (size_t)(n > 1 ? n : 1));
    int64_t m = 0;
    for (int64_t u = 0; u < n; ++u) {
        if (u == v) continue;
        uint64_t dd;
        if (po_dist2(theta + (int64_t)v * D, theta + u * D, D, &dd)) { free(all); return -1; }
        all[m].d2 = dd; all[m].id = (int32_t)u; ++m;
    }
    qsort(all, (size_t)m, sizeof(po_nb), po_cmp_nb);
    for (int i = 0; i < k; ++i) {
        if (i < m) { ids[i] = all[i].id; d2[i] = all[i].d2; }
        else { ids[i] = -1; d2[i] = UINT64_MAX; }
    }
    free(all);
    return 0;
}

/* ------------------------------------------------- all-core driver --- */
/* Each function below cuts one independent outer loop into nthreads
 * contiguous ranges and runs the single-threaded function on each range in a
 * thread of its own. Results are identical to the single-threaded call. */

typedef struct {
    int kind;
    int64_t a, b;                    /* range of this thread */
    /* shared arguments */
    int64_t n, R;
    int L, T, mode, k, D;
    const int64_t* row_ptr;
    const int32_t* col;
    const uint32_t* w;
    const uint64_t* thr_in;
    const int32_t* alias_in;
    const uint64_t* rowsum;
    uint64_t seed;
    const int32_t* paths;
    const int64_t* off;
    const int32_t* pidc;
    const int32_t* queries;
    /* outputs */
    uint64_t* thr;
    int32_t* alias;
    uint64_t* S;
    int32_t* out;
    int64_t* cnt;
    int32_t* pid;
    int32_t* ids;
    uint32_t* cnts;
    const uint32_t* theta;
    uint64_t* d2;
    const int64_t* rid;       /* JOB_PATHS_AT: path ids */
    const int32_t* qpos;      /* JOB_STREAM */
    uint64_t* cnt64;
    int64_t* npaths;
    int rc;
} po_job;

enum { JOB_ALIAS, JOB_ROWSUM, JOB_PATHS, JOB_IDX_COUNT, JOB_IDX_FILL, JOB_TOPK, JOB_THETA, JOB_KNN, JOB_PATHS_AT,
       JOB_STREAM };

static void* po_job_run(void* arg) {
    po_job* j = (po_job*)arg;
    j->rc = 0;
    switch (j->kind) {
    case JOB_ALIAS:
        for (int64_t v = j->a; v < j->b; ++v) {
            int64_t s = j->row_ptr[v], d = j->row_ptr[v + 1] - s;
            if (d > 0) po_alias_row(j->w + s, d, j->thr + s, j->alias + s);
        }
        break;
    case JOB_ROWSUM:
        po_row_sums(j->a, j->b, j->row_ptr, j->w, j->S);
        break;
    case JOB_PATHS:
        j->rc = po_sample_paths_rs(j->n, j->row_ptr, j->col, j->w, j->thr_in, j->alias_in, j->rowsum, j->seed,
                                   j->a, j->b, j->T, j->mode, j->out + (j->a - j->R) * (j->T + 1));
        break;
    case JOB_IDX_COUNT:
        po_index_range(j->R, j->L, j->paths, j->a, j->b, j->cnt, NULL);
        break;
    case JOB_IDX_FILL:
        po_index_range(j->R, j->L, j->paths, j->a, j->b, j->cnt, j->pid);
        break;
    case JOB_PATHS_AT:
        for (int64_t i = j->a; i < j->b && !j->rc; ++i)
            j->rc = po_sample_paths_rs(j->n, j->row_ptr, j->col, j->w, j->thr_in, j->alias_in, j->rowsum, j->seed,
                                       j->rid[i], j->rid[i] + 1, j->T, j->mode, j->out + i * (j->T + 1));
        break;
    case JOB_STREAM:
        j->rc = po_stream_counts(j->n, j->row_ptr, j->col, j->w, j->thr_in, j->alias_in, j->rowsum, j->seed, j->a,
                                 j->b, j->T, j->mode, j->qpos, j->cnt64, j->npaths);
        break;
    case JOB_KNN:
        for (int64_t i = j->a; i < j->b; ++i)
            if (po_knn(j->n, j->D, j->theta, j->queries[i], j->k, j->ids + i * j->k, j->d2 + i * j->k)) j->rc = -1;
        break;
    case JOB_TOPK:
    case JOB_THETA: {
        /* zeroed up front (not lazily by calloc), so every call pays the
           same fixed cost whatever its queries touch */
        size_t wbytes = sizeof(uint32_t) * (size_t)(j->n > 0 ? j->n : 1);
        uint32_t* work = (uint32_t*)malloc(wbytes);
        if (!work) { j->rc = -1; break; }
        memset(work, 0, wbytes);
        for (int64_t i = j->a; i < j->b; ++i) {
            int32_t v = j->queries ? j->queries[i] : (int32_t)i;
            if (j->kind == JOB_TOPK)
                po_topk(j->n, j->L, j->paths, j->off, j->pidc, v, j->k, work, j->ids + i * j->k, j->cnts + i * j->k);
            else
                po_theta(j->n, j->L, j->paths, j->off, j->pidc, v, j->D, work, j->cnts + i * j->D);
        }
        free(work);
        break;
    }
    }
    return NULL;
}

/* run `proto` on nthreads ranges whose bounds are cut[0..nthreads] */
static int po_run_ranges(const po_job* proto, int nthreads, const int64_t* cut) {
    po_job* jobs = (po_job*)malloc(sizeof(po_job) * (size_t)nthreads);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    int rc = 0;
    if (!jobs || !th) { free(jobs); free(th); return -1; }
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *proto;
        jobs[t].a = cut[t];
        jobs[t].b = cut[t + 1];
        if (pthread_create(&th[t], NULL, po_job_run, &jobs[t]) != 0) { jobs[t].rc = -1; th[t] = 0; }
    }
    for (int t = 0; t < nthreads; ++t) {
        if (th[t]) pthread_join(th[t], NULL);
        else po_job_run(&jobs[t]);             /* no thread: run the range here */
        if (jobs[t].rc) rc = jobs[t].rc;
    }
    free(jobs);
    free(th);
    return rc;
}

/* equal ranges of [lo, hi) */
static void po_cut_even(int64_t lo, int64_t hi, int nthreads, int64_t* cut) {
    for (int t = 0; t <= nthreads; ++t) cut[t] = lo + (hi - lo) * t / nthreads;
}

/* row ranges holding about equal numbers of CSR entries */
static void po_cut_rows(int64_t n, const int64_t* row_ptr, int nthreads, int64_t* cut) {
    int64_t m = row_ptr[n], v = 0;
    cut[0] = 0;
    for (int t = 1; t < nthreads; ++t) {
        int64_t target = m * t / nthreads;
        while (v < n && row_ptr[v] < target) ++v;
        cut[t] = v;
    }
    cut[nthreads] = n;
}

int po_mt_alias_tables(int64_t n, const int64_t* row_ptr, const uint32_t* w, uint64_t* thr, int32_t* alias,
                       int nthreads) {
    if (nthreads < 1) nthreads = 1;
    int64_t* cut = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nthreads + 1));
    po_job j;
    memset(&j, 0, sizeof j);
    j.kind = JOB_ALIAS; j.row_ptr = row_ptr; j.w = w; j.thr = thr; j.alias = alias;
    po_cut_rows(n, row_ptr, nthreads, cut);
    int rc = po_run_ranges(&j, nthreads, cut);
    free(cut);
    return rc;
}

/* Paths r0..r1-1 as po_sample_paths (S_v summed once per row first). */
int po_mt_sample_paths(int64_t n, const int64_t* row_ptr, const int32_t* col, const uint32_t* w,
                       const uint64_t* thr, const int32_t* alias, uint64_t seed, int64_t r0, int64_t r1, int T,
                       int mode, int32_t* out, int nthreads) {
    if (n < 1 || T < 0 || T > 65535 || (mode != 0 && mode != 1) || r1 < r0) return -1;
    if (nthreads < 1) nthreads = 1;
    int64_t* cut = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nthreads + 1));
    uint64_t* S = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    if (!cut || !S) { free(cut); free(S); return -1; }
    po_job j;
    memset(&j, 0, sizeof j);
    j.kind = JOB_ROWSUM; j.row_ptr = row_ptr; j.w = w; j.S = S;
    po_cut_rows(n, row_ptr, nthreads, cut);
    int rc = po_run_ranges(&j, nthreads, cut);
    if (!rc) {
        memset(&j, 0, sizeof j);
        j.kind = JOB_PATHS; j.n = n; j.row_ptr = row_ptr; j.col = col; j.w = w; j.thr_in = thr; j.alias_in = alias;
        j.rowsum = S; j.seed = seed; j.T = T; j.mode = mode; j.out = out;
        j.R = r0;                            /* row of path r is r - r0 */
        po_cut_even(r0, r1, nthreads, cut);
        rc = po_run_ranges(&j, nthreads, cut);
    }
    free(S);
    free(cut);
    return rc;
}

/* po_build_index with one vertex range per thread (off and pid as there). */
int64_t po_mt_build_index(int64_t n, int64_t R, int L, const int32_t* paths, int64_t* off, int32_t* pid,
                          int nthreads) {
    if (nthreads < 1) nthreads = 1;
    int64_t* cut = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nthreads + 1));
    if (!cut) return -1;
    po_cut_even(0, n, nthreads, cut);
    memset(off, 0, sizeof(int64_t) * (size_t)(n + 1));
    po_job j;
    memset(&j, 0, sizeof j);
    j.R = R; j.L = L; j.paths = paths;
    /* counts: thread t writes |P_v| to off[v + 1] for its vertices */
    j.kind = JOB_IDX_COUNT;
    j.cnt = off + 1;                       /* po_index_range indexes cnt[u - v0]: shift per range below */
    po_job* jobs = (po_job*)malloc(sizeof(po_job) * (size_t)nthreads);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    int64_t* cur = pid ? (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1)) : NULL;
    if (!jobs || !th || (pid && !cur)) { free(jobs); free(th); free(cur); free(cut); return -1; }
    for (int pass = 0; pass < (pid ? 2 : 1); ++pass) {
        for (int t = 0; t < nthreads; ++t) {
            jobs[t] = j;
            jobs[t].a = cut[t];
            jobs[t].b = cut[t + 1];
            jobs[t].kind = pass ? JOB_IDX_FILL : JOB_IDX_COUNT;
            jobs[t].cnt = pass ? cur + cut[t] : off + 1 + cut[t];
            jobs[t].pid = pass ? pid : NULL;
            if (pthread_create(&th[t], NULL, po_job_run, &jobs[t]) != 0) th[t] = 0;
        }
        for (int t = 0; t < nthreads; ++t) {
            if (th[t]) pthread_join(th[t], NULL);
            else po_job_run(&jobs[t]);
        }
        if (pass == 0) {
            for (int64_t v = 0; v < n; ++v) off[v + 1] += off[v];
            if (cur) memcpy(cur, off, sizeof(int64_t) * (size_t)n);
        }
    }
    free(jobs);
    free(th);
    free(cur);
    free(cut);
    return off[n];
}

/* po_topk for queries[0..q) (NULL: vertices 0..q-1), rows ids[q][k], cnts[q][k]. */
int po_mt_topk_many(int64_t n, int L, const int32_t* paths, const int64_t* off, const int32_t* pid,
                    const int32_t* queries, int64_t q, int k, int32_t* ids, uint32_t* cnts, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    int64_t* cut = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nthreads + 1));
    if (!cut) return -1;
    po_job j;
    memset(&j, 0, sizeof j);
    j.kind = JOB_TOPK; j.n = n; j.L = L; j.paths = paths; j.off = off; j.pidc = pid; j.queries = queries;
    j.k = k; j.ids = ids; j.cnts = cnts;
    po_cut_even(0, q, nthreads, cut);
    int rc = po_run_ranges(&j, nthreads, cut);
    free(cut);
    return rc;
}

/* po_theta for queries[0..q) (NULL: vertices 0..q-1), rows theta[q][D]. */
int po_mt_theta_many(int64_t n, int L, const int32_t* paths, const int64_t* off, const int32_t* pid,
                     const int32_t* queries, int64_t q, int D, uint32_t* theta, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    int64_t* cut = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nthreads + 1));
    if (!cut) return -1;
    po_job j;
    memset(&j, 0, sizeof j);
    j.kind = JOB_THETA; j.n = n; j.L = L; j.paths = paths; j.off = off; j.pidc = pid; j.queries = queries;
    j.D = D; j.cnts = theta;
    po_cut_even(0, q, nthreads, cut);
    int rc = po_run_ranges(&j, nthreads, cut);
    free(cut);
    return rc;
}

/* po_knn for queries[0..q), rows ids[q][k], d2[q][k]; -1 if a distance overflows. */
int po_mt_knn_many(int64_t n, int D, const uint32_t* theta, const int32_t* queries, int64_t q, int k, int32_t* ids,
                   uint64_t* d2, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    int64_t* cut = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nthreads + 1));
    if (!cut) return -1;
    po_job j;
    memset(&j, 0, sizeof j);
    j.kind = JOB_KNN; j.n = n; j.D = D; j.theta = theta; j.queries = queries; j.k = k; j.ids = ids; j.d2 = d2;
    po_cut_even(0, q, nthreads, cut);
    int rc = po_run_ranges(&j, nthreads, cut);
    free(cut);
    return rc;
}

/* S_v of every row on nthreads row ranges (malloc'd; NULL on failure) */
static uint64_t* po_mt_row_sums(int64_t n, const int64_t* row_ptr, const uint32_t* w, int nthreads) {
    int64_t* cut = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nthreads + 1));
    uint64_t* S = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    if (!cut || !S) { free(cut); free(S); return NULL; }
    po_job j;
    memset(&j, 0, sizeof j);
    j.kind = JOB_ROWSUM; j.row_ptr = row_ptr; j.w = w; j.S = S;
    po_cut_rows(n, row_ptr, nthreads, cut);
    int rc = po_run_ranges(&j, nthreads, cut);
    free(cut);
    if (rc) { free(S); return NULL; }
    return S;
}

/* Paths ids[0..m) (any order, repeats allowed) as po_sample_paths draws
 * them: row i of out (int32[m][T+1]) is path ids[i]. */
int po_mt_paths_at(int64_t n, const int64_t* row_ptr, const int32_t* col, const uint32_t* w, const uint64_t* thr,
                   const int32_t* alias, uint64_t seed, const int64_t* ids, int64_t m, int T, int mode, int32_t* out,
                   int nthreads) {
    if (n < 1 || T < 0 || T > 65535 || (mode != 0 && mode != 1) || m < 0) return -1;
    for (int64_t i = 0; i < m; ++i) if (ids[i] < 0) return -1;
    if (nthreads < 1) nthreads = 1;
    uint64_t* S = po_mt_row_sums(n, row_ptr, w, nthreads);
    int64_t* cut = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nthreads + 1));
    if (!S || !cut) { free(S); free(cut); return -1; }
    po_job j;
    memset(&j, 0, sizeof j);
    j.kind = JOB_PATHS_AT; j.n = n; j.row_ptr = row_ptr; j.col = col; j.w = w; j.thr_in = thr; j.alias_in = alias;
    j.rowsum = S; j.seed = seed; j.T = T; j.mode = mode; j.out = out; j.rid = ids;
    po_cut_even(0, m, nthreads, cut);
    int rc = po_run_ranges(&j, nthreads, cut);
    free(S);
    free(cut);
    return rc;
}

/* po_stream_counts over paths r0..r1-1 for the distinct vertices
 * queries[0..nq): each thread takes one contiguous range of path ids with
 * counters of its own, which are then added up (sums do not depend on the
 * split). cnt is uint64[nq][n] and npaths int64[n], both overwritten. */
int po_mt_stream_counts(int64_t n, const int64_t* row_ptr, const int32_t* col, const uint32_t* w,
                        const uint64_t* thr, const int32_t* alias, uint64_t seed, int64_t r0, int64_t r1, int T,
                        int mode, const int32_t* queries, int64_t nq, uint64_t* cnt, int64_t* npaths, int nthreads) {
    if (n < 1 || T < 0 || T > 65535 || (mode != 0 && mode != 1) || r1 < r0 || nq < 0) return -1;
    if (nthreads < 1) nthreads = 1;
    int32_t* qpos = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!qpos) return -1;
    for (int64_t v = 0; v < n; ++v) qpos[v] = -1;
    for (int64_t i = 0; i < nq; ++i) {
        if (queries[i] < 0 || queries[i] >= n || qpos[queries[i]] >= 0) { free(qpos); return -1; }
        qpos[queries[i]] = (int32_t)i;
    }
    size_t ncnt = (size_t)nq * (size_t)n;
    uint64_t* S = po_mt_row_sums(n, row_ptr, w, nthreads);
    int64_t* cut = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nthreads + 1));
    po_job* jobs = (po_job*)malloc(sizeof(po_job) * (size_t)nthreads);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    uint64_t* tc = (uint64_t*)malloc(sizeof(uint64_t) * (ncnt > 0 ? ncnt : 1) * (size_t)nthreads);
    int64_t* tn = (int64_t*)malloc(sizeof(int64_t) * (size_t)n * (size_t)nthreads);
    int rc = 0;
    if (!S || !cut || !jobs || !th || !tc || !tn) rc = -1;
    if (!rc) {
        memset(tc, 0, sizeof(uint64_t) * (ncnt > 0 ? ncnt : 1) * (size_t)nthreads);
        memset(tn, 0, sizeof(int64_t) * (size_t)n * (size_t)nthreads);
        po_cut_even(r0, r1, nthreads, cut);
        for (int t = 0; t < nthreads; ++t) {
            memset(&jobs[t], 0, sizeof(po_job));
            jobs[t].kind = JOB_STREAM; jobs[t].n = n; jobs[t].row_ptr = row_ptr; jobs[t].col = col; jobs[t].w = w;
            jobs[t].thr_in = thr; jobs[t].alias_in = alias; jobs[t].rowsum = S; jobs[t].seed = seed;
            jobs[t].T = T; jobs[t].mode = mode; jobs[t].qpos = qpos;
            jobs[t].a = cut[t]; jobs[t].b = cut[t + 1];
            jobs[t].cnt64 = tc + (size_t)t * (ncnt > 0 ? ncnt : 1);
            jobs[t].npaths = tn + (size_t)t * (size_t)n;
            if (pthread_create(&th[t], NULL, po_job_run, &jobs[t]) != 0) th[t] = 0;
        }
        for (int t = 0; t < nthreads; ++t) {
            if (th[t]) pthread_join(th[t], NULL);
            else po_job_run(&jobs[t]);
            if (jobs[t].rc) rc = jobs[t].rc;
        }
    }
    if (!rc) {
        memset(cnt, 0, sizeof(uint64_t) * ncnt);
        memset(npaths, 0, sizeof(int64_t) * (size_t)n);
        for (int t = 0; t < nthreads; ++t) {
            const uint64_t* c = tc + (size_t)t * (ncnt > 0 ? ncnt : 1);
            const int64_t* m = tn + (size_t)t * (size_t)n;
            for (size_t i = 0; i < ncnt; ++i) cnt[i] += c[i];
            for (int64_t v = 0; v < n; ++v) npaths[v] += m[v];
        }
    }
    free(qpos); free(S); free(cut); free(jobs); free(th); free(tc); free(tn);
    return rc;
}
