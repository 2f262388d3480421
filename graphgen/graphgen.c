/*
 * graphgen.c -- seeded synthetic graph generators (edge tuples only).
 *
 * This file produces raw (src, dst) vertex-id tuples.  It holds no triangle
 * counting arithmetic and no CSR construction: symmetrising, dropping
 * self-loops, de-duplicating and sorting are the job of the code that consumes
 * the tuples (the CPU oracle does it its own way, the CUDA library its own
 * way).  Both sides call these functions so that they see the same input.
 *
 * Randomness: every draw is SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator: draw(key, i) = mix(key + (i + 1) * golden), with
 * key = mix(seed * golden ^ stream_tag).  A draw depends only on (seed,
 * stream, index), so the parallel loops below give the same output for any
 * thread count.
 *
 * Families (shapes of the workloads in the paper's experiments section and the
 * configurations of this library's benchmarks):
 *   - R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with Graph500-style
 *     quadrant probabilities and an optional seeded vertex permutation;
 *   - Erdos-Renyi G(n, m): exactly m distinct undirected loop-free pairs;
 *   - Chung-Lu power law (weights (i+1)^(-1/(gamma-1)) scaled to a target mean
 *     degree and capped at sqrt(sum w)), endpoints drawn with Vose's alias
 *     method;
 *   - a road-like R x C grid with one random diagonal per cell with
 *     probability p (triangle count 2 * #diagonals, a closed form).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GG_GOLDEN 0x9E3779B97F4A7C15ULL

enum {
    GG_STREAM_RMAT = 0x524D4154u,   /* quadrant draws */
    GG_STREAM_PERM = 0x5045524Du,   /* vertex permutation */
    GG_STREAM_ER = 0x45524552u,     /* Erdos-Renyi endpoints */
    GG_STREAM_CL = 0x43484C55u,     /* Chung-Lu endpoints */
    GG_STREAM_GRID = 0x47524944u,   /* grid diagonals */
};

static inline uint64_t gg_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t gg_key(uint64_t seed, uint32_t stream)
{
    return gg_mix(seed * GG_GOLDEN ^ (uint64_t)stream);
}

static inline uint64_t gg_draw(uint64_t key, uint64_t i)
{
    return gg_mix(key + (i + 1) * GG_GOLDEN);
}

/* Uniform integer in [0, bound) from a 64-bit draw (multiply-shift; the bias
 * is below 2^-32 for bound < 2^32). */
static inline uint32_t gg_below(uint64_t r, uint32_t bound)
{
    return (uint32_t)(((r >> 32) * (uint64_t)bound) >> 32);
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double gg_unit(uint64_t r)
{
    return (double)(r >> 11) * (1.0 / 9007199254740992.0);
}

/* Seeded uniformly random permutation of 0..n-1 (Fisher-Yates from the top,
 * step i draws j in [0, i]). */
void gg_permutation(uint32_t n, uint64_t seed, uint32_t *perm)
{
    const uint64_t key = gg_key(seed, GG_STREAM_PERM);
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    for (uint32_t i = n; i > 1; --i) {
        uint32_t j = gg_below(gg_draw(key, i - 1), i);
        uint32_t t = perm[i - 1];
        perm[i - 1] = perm[j];
        perm[j] = t;
    }
}

/*
 * R-MAT tuples.  Tuple t draws `scale` quadrants; quadrant q at bit position
 * `scale-1-l` uses 32 random bits: q = 0 (a) if x < ta, 1 (b: column bit) if
 * x < tb, 2 (c: row bit) if x < tc, else 3 (d: both bits), where ta, tb, tc are
 * the cumulative probabilities scaled to 2^32.  With permute != 0 both
 * endpoints go through gg_permutation(2^scale, seed).
 */
void gg_rmat(int scale, uint64_t n_tuples, uint32_t ta, uint32_t tb, uint32_t tc,
             uint64_t seed, int permute, uint32_t *src, uint32_t *dst)
{
    const uint64_t key = gg_key(seed, GG_STREAM_RMAT);
    const uint32_t pairs = (uint32_t)((scale + 1) / 2);
    const uint32_t n = 1u << scale;
    uint32_t *perm = NULL;
    if (permute) {
        perm = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
        gg_permutation(n, seed, perm);
    }
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < (int64_t)n_tuples; ++t) {
        uint32_t u = 0, v = 0;
        for (uint32_t p = 0; p < pairs; ++p) {
            uint64_t r = gg_draw(key, (uint64_t)t * pairs + p);
            for (int half = 0; half < 2; ++half) {
                int l = (int)(2 * p + (uint32_t)half);
                if (l >= scale) break;
                uint32_t x = half ? (uint32_t)r : (uint32_t)(r >> 32);
                uint32_t bit = 1u << (scale - 1 - l);
                if (x < ta) {
                } else if (x < tb) {
                    v |= bit;
                } else if (x < tc) {
                    u |= bit;
                } else {
                    u |= bit;
                    v |= bit;
                }
            }
        }
        if (perm) {
            u = perm[u];
            v = perm[v];
        }
        src[t] = u;
        dst[t] = v;
    }
    free(perm);
}

/*
 * Erdos-Renyi G(n, m): m distinct unordered pairs {a, b}, a != b, written as
 * (min, max).  Candidates are drawn in index order (two endpoint draws per
 * candidate), loops are rejected and repeats are rejected through an
 * open-addressing set, until m pairs are kept.  Returns the number written
 * (m, or fewer only when m exceeds n(n-1)/2).
 */
uint64_t gg_er(uint32_t n, uint64_t m, uint64_t seed, uint32_t *src, uint32_t *dst)
{
    if (n < 2) return 0;
    const uint64_t max_pairs = (uint64_t)n * (n - 1) / 2;
    if (m > max_pairs) m = max_pairs;
    uint64_t cap = 16;
    while (cap < 2 * m + 16) cap <<= 1;
    uint64_t *set = (uint64_t *)malloc(sizeof(uint64_t) * cap);
    memset(set, 0xFF, sizeof(uint64_t) * cap);
    const uint64_t key = gg_key(seed, GG_STREAM_ER);
    uint64_t kept = 0;
    for (uint64_t i = 0; kept < m; ++i) {
        uint32_t a = gg_below(gg_draw(key, 2 * i), n);
        uint32_t b = gg_below(gg_draw(key, 2 * i + 1), n);
        if (a == b) continue;
        if (a > b) { uint32_t t = a; a = b; b = t; }
        uint64_t k = ((uint64_t)a << 32) | b;
        uint64_t h = gg_mix(k) & (cap - 1);
        int fresh = 1;
        while (set[h] != UINT64_MAX) {
            if (set[h] == k) { fresh = 0; break; }
            h = (h + 1) & (cap - 1);
        }
        if (!fresh) continue;
        set[h] = k;
        src[kept] = a;
        dst[kept] = b;
        ++kept;
    }
    free(set);
    return kept;
}

/*
 * Chung-Lu tuples.  Weight of vertex i: w_i = (i+1)^(-1/(gamma-1)), scaled so
 * that sum w = mean_deg * n, then capped at sqrt(sum w) (sum taken after
 * scaling, before capping).  Each tuple draws both endpoints independently
 * with probability proportional to the capped weights (Vose's alias method,
 * two draws per endpoint: column, coin).  With permute != 0 vertex ids go
 * through gg_permutation(n, seed).  stats[0] = sum of capped weights,
 * stats[1] = largest capped weight.
 */
void gg_chung_lu(uint32_t n, double gamma, double mean_deg, uint64_t n_tuples, uint64_t seed,
                 int permute, uint32_t *src, uint32_t *dst, double *stats)
{
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double s = 0.0;
    const double ex = -1.0 / (gamma - 1.0);
    for (uint32_t i = 0; i < n; ++i) {
        w[i] = pow((double)i + 1.0, ex);
        s += w[i];
    }
    const double scale = mean_deg * (double)n / s;
    const double cap = sqrt(mean_deg * (double)n);
    double total = 0.0, wmax = 0.0;
    for (uint32_t i = 0; i < n; ++i) {
        w[i] *= scale;
        if (w[i] > cap) w[i] = cap;
        total += w[i];
        if (w[i] > wmax) wmax = w[i];
    }
    if (stats) {
        stats[0] = total;
        stats[1] = wmax;
    }
    /* Vose's alias table over the normalised weights. */
    double *prob = (double *)malloc(sizeof(double) * (size_t)n);
    uint32_t *alias = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    uint32_t *small = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    uint32_t *large = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    uint32_t ns = 0, nl = 0;
    for (uint32_t i = 0; i < n; ++i) {
        prob[i] = w[i] * (double)n / total;
        if (prob[i] < 1.0) small[ns++] = i; else large[nl++] = i;
    }
    while (ns > 0 && nl > 0) {
        uint32_t l = small[--ns], g = large[--nl];
        alias[l] = g;
        prob[g] = (prob[g] + prob[l]) - 1.0;
        if (prob[g] < 1.0) small[ns++] = g; else large[nl++] = g;
    }
    while (nl > 0) { uint32_t g = large[--nl]; prob[g] = 1.0; alias[g] = g; }
    while (ns > 0) { uint32_t l = small[--ns]; prob[l] = 1.0; alias[l] = l; }
    free(small);
    free(large);
    uint32_t *perm = NULL;
    if (permute) {
        perm = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
        gg_permutation(n, seed, perm);
    }
    const uint64_t key = gg_key(seed, GG_STREAM_CL);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < (int64_t)n_tuples; ++t) {
        uint32_t e[2];
        for (int k = 0; k < 2; ++k) {
            uint64_t base = ((uint64_t)t * 2 + (uint64_t)k) * 2;
            uint32_t col = gg_below(gg_draw(key, base), n);
            double coin = gg_unit(gg_draw(key, base + 1));
            e[k] = coin < prob[col] ? col : alias[col];
            if (perm) e[k] = perm[e[k]];
        }
        src[t] = e[0];
        dst[t] = e[1];
    }
    free(perm);
    free(prob);
    free(alias);
    free(w);
}

/*
 * R x C grid (vertex (r, c) has id r*C + c): right and down edges, then for
 * every cell (r, c) (r < R-1, c < C-1) with probability p one diagonal, either
 * (r,c)-(r+1,c+1) or (r,c+1)-(r+1,c) by a fair coin.  Writes the tuples
 * (grid edges first, then diagonals in cell order) and returns their number;
 * *n_diag receives the diagonal count.  Capacity needed:
 * R*(C-1) + (R-1)*C + (R-1)*(C-1).
 */
uint64_t gg_grid(uint32_t R, uint32_t C, double p, uint64_t seed, uint32_t *src, uint32_t *dst,
                 uint64_t *n_diag)
{
    uint64_t k = 0;
    for (uint32_t r = 0; r < R; ++r)
        for (uint32_t c = 0; c + 1 < C; ++c) {
            src[k] = r * C + c;
            dst[k] = r * C + c + 1;
            ++k;
        }
    for (uint32_t r = 0; r + 1 < R; ++r)
        for (uint32_t c = 0; c < C; ++c) {
            src[k] = r * C + c;
            dst[k] = (r + 1) * C + c;
            ++k;
        }
    const uint64_t key = gg_key(seed, GG_STREAM_GRID);
    const uint64_t thr = (uint64_t)(p * 4294967296.0);
    uint64_t d = 0;
    for (uint32_t r = 0; r + 1 < R; ++r)
        for (uint32_t c = 0; c + 1 < C; ++c) {
            uint64_t cell = (uint64_t)r * (C - 1) + c;
            uint64_t x = gg_draw(key, cell);
            if ((x >> 32) >= thr) continue;
            if (x & 1) {
                src[k] = r * C + c;
                dst[k] = (r + 1) * C + c + 1;
            } else {
                src[k] = r * C + c + 1;
                dst[k] = (r + 1) * C + c;
            }
            ++k;
            ++d;
        }
    if (n_diag) *n_diag = d;
    return k;
}

/* Raw SplitMix64 draws, exposed for tests of the generator itself. */
void gg_draws(uint64_t seed, uint32_t stream, uint64_t first, uint64_t count, uint64_t *out)
{
    const uint64_t key = gg_key(seed, stream);
    for (uint64_t i = 0; i < count; ++i) out[i] = gg_draw(key, first + i);
}
