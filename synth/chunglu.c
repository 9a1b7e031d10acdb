/*
 * Seeded synthetic inputs: Chung-Lu power-law graphs and query mixes.
 *
 * This module produces INPUTS only. It holds none of the method's arithmetic
 * (no path sampling, no selection, no counting) and shares no code with either
 * the CUDA path or the CPU oracle; both read the CSR arrays it writes.
 *
 * Graph recipe (ball-dropping Chung-Lu, "first E distinct edges"):
 *   - target weights  omega_i = (i+1)^(-1/(gamma-1)),  i in [0, n)
 *   - integer weights W_i = max(1, floor(omega_i * 2^32)); an integer Vose
 *     alias table over W picks each endpoint of a draw
 *   - draw d (d = 0, 1, 2, ...) gives endpoints (a, b) from four SplitMix64
 *     words keyed by (seed, stream 0x47, 4d..4d+3); self-loops are dropped
 *   - the graph is the first E = n*mean_deg/2 distinct undirected edges in
 *     draw order (a pure function of the infinite draw sequence, so the batch
 *     size used internally does not change the result)
 *   - edge weight = f(SplitMix64(seed, stream 0x57, (min<<32)|max)): it
 *     depends only on the endpoints; uniform [lo,hi] or log-uniform [1,hi]
 *   - output: symmetric CSR, columns ascending in every row, no self-loops
 *
 * Transcendentals use det_log/det_exp below, built from + - * / and the exact
 * frexp/ldexp only (compiled with -ffp-contract=off), so the same graph comes
 * out on every IEEE-754 machine (x86-64 here, aarch64 on the GPU host).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <omp.h>

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------- RNG --- */
/* SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014), used as a
 * counter-based hash: out = mix(key + (ctr+1) * golden). */
static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static inline uint64_t sm64(uint64_t key, uint64_t ctr) {
    return sm64_mix(key + (ctr + 1) * 0x9E3779B97F4A7C15ULL);
}
static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return sm64_mix(sm64_mix(seed ^ 0x5EED5EED5EED5EEDULL) + stream * 0xD1B54A32D192ED03ULL);
}
static inline uint64_t mulhi(uint64_t a, uint64_t b) { return (uint64_t)(((u128)a * b) >> 64); }

/* ------------------------------------------------ deterministic log/exp --- */
static const double LN2 = 0.69314718055994530942;
static double det_log(double x) {
    int e; double m = frexp(x, &e);             /* x = m*2^e, m in [0.5,1) */
    if (m < 0.70710678118654752440) { m *= 2.0; e -= 1; }
    double s = (m - 1.0) / (m + 1.0), s2 = s * s, t = s, sum = 0.0;
    for (int k = 0; k < 16; ++k) { sum += t / (double)(2 * k + 1); t *= s2; }
    return 2.0 * sum + (double)e * LN2;
}
static double det_exp(double x) {
    double kf = floor(x / LN2 + 0.5);
    double r = x - kf * LN2;                     /* |r| <= ~ln2/2 */
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 24; ++k) { term *= r / (double)k; sum += term; }
    return ldexp(sum, (int)kf);
}
double synth_det_pow(double b, double e) { return det_exp(e * det_log(b)); }

/* ------------------------------------------------------ parallel radix --- */
/* Stable LSD radix sort of 64-bit keys (optionally with a uint32 payload). */
#define RBITS 11
#define RBUCK (1 << RBITS)
static void radix_sort(uint64_t* k0, uint32_t* v0, int64_t n, int key_bits,
                       uint64_t* tk0, uint32_t* tv0) {
    int nt = omp_get_max_threads();
    int64_t* hist = (int64_t*)malloc(sizeof(int64_t) * (size_t)nt * RBUCK);
    uint64_t *k = k0, *tk = tk0;
    uint32_t *v = v0, *tv = tv0;
    int passes = 0;
    for (int shift = 0; shift < key_bits; shift += RBITS) {
        memset(hist, 0, sizeof(int64_t) * (size_t)nt * RBUCK);
        #pragma omp parallel num_threads(nt)
        {
            int t = omp_get_thread_num();
            int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
            int64_t* h = hist + (size_t)t * RBUCK;
            for (int64_t i = lo; i < hi; ++i) h[(k[i] >> shift) & (RBUCK - 1)]++;
            #pragma omp barrier
            #pragma omp single
            {
                int64_t run = 0;
                for (int d = 0; d < RBUCK; ++d)
                    for (int tt = 0; tt < nt; ++tt) {
                        int64_t c = hist[(size_t)tt * RBUCK + d];
                        hist[(size_t)tt * RBUCK + d] = run; run += c;
                    }
            }
            for (int64_t i = lo; i < hi; ++i) {
                int64_t p = h[(k[i] >> shift) & (RBUCK - 1)]++;
                tk[p] = k[i];
                if (v) tv[p] = v[i];
            }
        }
        uint64_t* sk = k; k = tk; tk = sk;
        uint32_t* sv = v; v = tv; tv = sv;
        ++passes;
    }
    if (passes & 1) {   /* sorted data sits in the temporary buffers */
        memcpy(k0, k, sizeof(uint64_t) * (size_t)n);
        if (v0) memcpy(v0, v, sizeof(uint32_t) * (size_t)n);
    }
    free(hist);
}

static int bits_for(uint64_t x) { int b = 1; while ((1ULL << b) <= x && b < 63) ++b; return b; }

/* ------------------------------------------------------------ alias pick --- */
typedef struct { uint64_t thr; uint32_t alias; } vert_alias;

static void build_vertex_alias(int64_t n, const uint64_t* W, vert_alias* tab, uint64_t* total_out) {
    uint64_t total = 0;
    for (int64_t i = 0; i < n; ++i) total += W[i];
    /* q_i = W_i * n against capacity 'total' per column */
    uint64_t* q = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    int64_t* small = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t* large = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < n; ++i) {
        q[i] = W[i] * (uint64_t)n;
        if (q[i] < total) small[ns++] = i; else large[nl++] = i;
    }
    while (ns > 0 && nl > 0) {
        int64_t s = small[--ns], l = large[--nl];
        tab[s].thr = q[s]; tab[s].alias = (uint32_t)l;
        q[l] -= total - q[s];
        if (q[l] < total) small[ns++] = l; else large[nl++] = l;
    }
    while (nl > 0) { int64_t l = large[--nl]; tab[l].thr = total; tab[l].alias = (uint32_t)l; }
    while (ns > 0) { int64_t s = small[--ns]; tab[s].thr = total; tab[s].alias = (uint32_t)s; }
    free(q); free(small); free(large);
    *total_out = total;
}
static inline uint32_t pick(const vert_alias* tab, int64_t n, uint64_t total, uint64_t x, uint64_t y) {
    uint64_t c = mulhi(x, (uint64_t)n);
    uint64_t u = mulhi(y, total);
    return u < tab[c].thr ? (uint32_t)c : tab[c].alias;
}

/* --------------------------------------------------------- edge weight --- */
static inline uint32_t edge_weight(uint64_t wkey, uint64_t a, uint64_t b, int wkind,
                                   uint32_t lo, uint32_t hi, double lnhi1) {
    uint64_t h = sm64(wkey, (a << 32) | b);
    if (wkind == 0) return lo + (uint32_t)mulhi(h, (uint64_t)(hi - lo) + 1);
    /* log-uniform on [1, hi]: floor((hi+1)^u) clamped to [1, hi] */
    double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
    double x = floor(det_exp(u * lnhi1));
    if (x < 1.0) x = 1.0;
    if (x > (double)hi) x = (double)hi;
    return (uint32_t)x;
}

/*
 * Generate the graph. Returns 0 on success, negative on error.
 * row_ptr[n+1], col[2E], w[2E] are caller-allocated with E = n*mean_deg/2.
 * stats[0] = draws used, stats[1] = max degree, stats[2] = isolated vertices.
 */
int synth_chung_lu(int64_t n, int64_t E, double gamma, uint64_t seed,
                   int wkind, uint32_t wlo, uint32_t whi,
                   int64_t* row_ptr, int32_t* col, uint32_t* w, int64_t* stats) {
    if (n < 2 || n > 0x7fffffff || E < 0 || gamma <= 1.0) return -1;
    if ((double)E > (double)n * (double)(n - 1) / 2.0 * 0.5) return -2;  /* too dense */
    if (whi < wlo || wlo < 1) return -3;
    double alpha = 1.0 / (gamma - 1.0);
    uint64_t* W = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double om = det_exp(-alpha * det_log((double)(i + 1)));
        double s = floor(om * 4294967296.0);
        W[i] = s < 1.0 ? 1 : (uint64_t)s;
    }
    vert_alias* tab = (vert_alias*)malloc(sizeof(vert_alias) * (size_t)n);
    uint64_t total;
    build_vertex_alias(n, W, tab, &total);
    free(W);

    uint64_t dkey = stream_key(seed, 0x47), wkey = stream_key(seed, 0x57);
    int vb = bits_for((uint64_t)n);
    int key_bits = 2 * vb;
    int64_t B = E + E / 8 + 1024;
    uint64_t *keys = NULL, *tk = NULL, *kept = NULL;
    uint32_t *idx = NULL, *tv = NULL;
    uint8_t* mark = NULL;
    int64_t nkept = 0;
    for (int attempt = 0; attempt < 12; ++attempt) {
        if (B > 0xffffffffLL) { free(tab); return -4; }
        keys = (uint64_t*)realloc(keys, sizeof(uint64_t) * (size_t)B);
        tk = (uint64_t*)realloc(tk, sizeof(uint64_t) * (size_t)B);
        idx = (uint32_t*)realloc(idx, sizeof(uint32_t) * (size_t)B);
        tv = (uint32_t*)realloc(tv, sizeof(uint32_t) * (size_t)B);
        int64_t m = 0;
        /* draws; self-loops get key UINT64_MAX (sorted to the end, ignored) */
        #pragma omp parallel for schedule(static)
        for (int64_t d = 0; d < B; ++d) {
            uint64_t c0 = 4 * (uint64_t)d;
            uint64_t a = pick(tab, n, total, sm64(dkey, c0), sm64(dkey, c0 + 1));
            uint64_t b = pick(tab, n, total, sm64(dkey, c0 + 2), sm64(dkey, c0 + 3));
            uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
            keys[d] = (a == b) ? (((1ULL << key_bits) - 1)) : ((lo << vb) | hi);
            idx[d] = (uint32_t)d;
        }
        radix_sort(keys, idx, B, key_bits, tk, tv);
        const uint64_t SELF = (1ULL << key_bits) - 1;
        /* first occurrence of each distinct key marks its draw index */
        mark = (uint8_t*)realloc(mark, (size_t)B);
        memset(mark, 0, (size_t)B);
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < B; ++i)
            if (keys[i] != SELF && (i == 0 || keys[i - 1] != keys[i])) mark[idx[i]] = 1;
        for (int64_t i = 0; i < B; ++i) m += mark[i];
        if (m < E) {
            double f = (double)E / (double)(m > 0 ? m : 1);
            B = (int64_t)((double)B * f * 1.15) + 4096;
            continue;
        }
        /* tau = draw index of the E-th distinct edge */
        int64_t cnt = 0, tau = -1;
        for (int64_t i = 0; i < B; ++i) { cnt += mark[i]; if (cnt == E) { tau = i; break; } }
        kept = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(E > 0 ? E : 1));
        for (int64_t i = 0; i < B; ++i)
            if (keys[i] != SELF && (i == 0 || keys[i - 1] != keys[i]) && (int64_t)idx[i] <= tau)
                kept[nkept++] = keys[i];
        stats[0] = tau + 1;
        break;
    }
    free(tab); free(idx); free(tv); free(mark);
    if (nkept != E) { free(keys); free(tk); free(kept); return -5; }

    /* swapped copy (max, min) sorted, for the lower part of every row */
    uint64_t* sw = keys;   /* reuse */
    const uint64_t vmask = (1ULL << vb) - 1;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < E; ++i) sw[i] = ((kept[i] & vmask) << vb) | (kept[i] >> vb);
    radix_sort(sw, NULL, E, key_bits, tk, NULL);
    free(tk);

    /* per-vertex ranges in both orders by binary search */
    int64_t* up = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t* dn = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    #pragma omp parallel for schedule(static)
    for (int64_t v = 0; v <= n; ++v) {
        uint64_t t = (uint64_t)v << vb;
        int64_t a = 0, b = E;
        while (a < b) { int64_t mid = (a + b) / 2; if (kept[mid] < t) a = mid + 1; else b = mid; }
        up[v] = a;
        a = 0; b = E;
        while (a < b) { int64_t mid = (a + b) / 2; if (sw[mid] < t) a = mid + 1; else b = mid; }
        dn[v] = a;
    }
    row_ptr[0] = 0;
    int64_t maxd = 0, iso = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t d = (up[v + 1] - up[v]) + (dn[v + 1] - dn[v]);
        row_ptr[v + 1] = row_ptr[v] + d;
        if (d > maxd) maxd = d;
        if (d == 0) ++iso;
    }
    double lnhi1 = det_log((double)whi + 1.0);
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < n; ++v) {
        int64_t p = row_ptr[v];
        for (int64_t i = dn[v]; i < dn[v + 1]; ++i) {       /* neighbours a < v */
            uint64_t a = sw[i] & vmask;
            col[p] = (int32_t)a; w[p] = edge_weight(wkey, a, (uint64_t)v, wkind, wlo, whi, lnhi1); ++p;
        }
        for (int64_t i = up[v]; i < up[v + 1]; ++i) {       /* neighbours b > v */
            uint64_t b = kept[i] & vmask;
            col[p] = (int32_t)b; w[p] = edge_weight(wkey, (uint64_t)v, b, wkind, wlo, whi, lnhi1); ++p;
        }
    }
    stats[1] = maxd; stats[2] = iso;
    free(up); free(dn); free(keys); free(kept);
    return 0;
}

/*
 * Query mix: nu uniform draws over [0,n) (with replacement) and nh uniform
 * draws over the hub set (the first ceil(0.01 n) vertices by (degree desc,
 * id asc)), then a Fisher-Yates shuffle of the concatenation. All words come
 * from SplitMix64 on stream 0x51. hubs[] is the caller-sorted hub list.
 */
void synth_query_mix(int64_t n, int64_t nu, const int32_t* hubs, int64_t nhubs, int64_t nh,
                     uint64_t seed, int32_t* out) {
    uint64_t k = stream_key(seed, 0x51);
    uint64_t c = 0;
    for (int64_t i = 0; i < nu; ++i) out[i] = (int32_t)mulhi(sm64(k, c++), (uint64_t)n);
    for (int64_t i = 0; i < nh; ++i) out[nu + i] = hubs[mulhi(sm64(k, c++), (uint64_t)nhubs)];
    for (int64_t i = nu + nh - 1; i > 0; --i) {
        int64_t j = (int64_t)mulhi(sm64(k, c++), (uint64_t)(i + 1));
        int32_t t = out[i]; out[i] = out[j]; out[j] = t;
    }
}

/* Uniform integer draws in [0, n) (test inputs such as random query lists). */
void synth_uniform_ints(int64_t count, int64_t n, uint64_t seed, uint64_t stream, int32_t* out) {
    uint64_t k = stream_key(seed, stream);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i) out[i] = (int32_t)mulhi(sm64(k, (uint64_t)i), (uint64_t)n);
}
