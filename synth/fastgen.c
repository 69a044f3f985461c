/*
 * fastgen.c -- multithreaded helpers of the seeded input generator (synth/).
 *
 * They reproduce exactly what synth/kb.py computes with numpy (same
 * counter-based SplitMix64 draws, same per-row duplicate redraws, same stable
 * transpose), so large knowledge bases can be generated in seconds.  Like the
 * rest of synth/, this code only makes inputs; it evaluates nothing.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ull

static inline uint64_t mix64(uint64_t x) {
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return mix64(mix64(seed * GOLDEN + 0x1234567ull) ^ (stream * 0xD1B54A32D192ED03ull));
}

static inline uint64_t draw(uint64_t key, uint64_t idx) { return mix64(key + (idx + 1) * GOLDEN); }

static inline uint32_t randint(uint64_t key, uint64_t idx, uint64_t hi) {
    return (uint32_t)((((draw(key, idx) >> 32)) * hi) >> 32);
}

static inline double uniform(uint64_t key, uint64_t idx) {
    return (double)(draw(key, idx) >> 11) * (1.0 / 9007199254740992.0);
}

static void sort_u32(uint32_t *a, int64_t n) {
    /* insertion sort for short rows, heap sort otherwise (rows can be long) */
    if (n < 32) {
        for (int64_t i = 1; i < n; ++i) {
            uint32_t v = a[i];
            int64_t j = i - 1;
            while (j >= 0 && a[j] > v) {
                a[j + 1] = a[j];
                --j;
            }
            a[j + 1] = v;
        }
        return;
    }
    for (int64_t start = n / 2 - 1; start >= 0; --start) {
        int64_t r = start;
        for (;;) {
            int64_t c = 2 * r + 1;
            if (c >= n) break;
            if (c + 1 < n && a[c + 1] > a[c]) ++c;
            if (a[r] >= a[c]) break;
            uint32_t t = a[r];
            a[r] = a[c];
            a[c] = t;
            r = c;
        }
    }
    for (int64_t end = n - 1; end > 0; --end) {
        uint32_t t = a[0];
        a[0] = a[end];
        a[end] = t;
        int64_t r = 0;
        for (;;) {
            int64_t c = 2 * r + 1;
            if (c >= end) break;
            if (c + 1 < end && a[c + 1] > a[c]) ++c;
            if (a[r] >= a[c]) break;
            t = a[r];
            a[r] = a[c];
            a[c] = t;
            r = c;
        }
    }
}

typedef struct {
    const uint64_t *rp;     /* [n+1] row offsets */
    int64_t r0, r1;         /* rows of this job */
    uint64_t n;
    uint64_t key_tgt, key_bias, key_pick;
    const uint8_t *smask;   /* subjects whose edges may be biased, or NULL */
    const int64_t *pool;
    int64_t pool_size;
    double pb;
    uint32_t *col;
    int64_t failed;
} targets_job;

static void *targets_worker(void *arg) {
    targets_job *j = (targets_job *)arg;
    for (int64_t i = j->r0; i < j->r1; ++i) {
        const uint64_t lo = j->rp[i], hi = j->rp[i + 1];
        uint32_t *row = j->col + lo;
        for (uint64_t k = lo; k < hi; ++k) {
            uint32_t t = randint(j->key_tgt, k, j->n);
            if (j->smask && j->smask[i] && j->pool_size > 0 && uniform(j->key_bias, k) < j->pb) {
                uint64_t pick = randint(j->key_pick, k, (uint64_t)j->pool_size);
                if ((int64_t)pick > j->pool_size - 1) pick = (uint64_t)(j->pool_size - 1);
                t = (uint32_t)j->pool[pick];
            }
            row[k - lo] = t;
        }
        const int64_t len = (int64_t)(hi - lo);
        sort_u32(row, len);
        for (uint64_t attempt = 1;; ++attempt) {
            int any = 0;
            /* positions whose value equals the previous one in the sorted row */
            for (int64_t q = len - 1; q >= 1; --q) {
                if (row[q] == row[q - 1]) {
                    row[q] = randint(j->key_tgt, lo + (uint64_t)q + attempt * (1ull << 40), j->n);
                    any = 1;
                }
            }
            if (!any) break;
            sort_u32(row, len);
            if (attempt > 10000) {
                j->failed = 1;
                break;
            }
        }
    }
    return NULL;
}

/* Draw the targets of one role (see synth/kb.py draw_targets). */
int fastgen_targets(uint64_t seed, uint64_t stream_tgt, uint64_t stream_bias, uint64_t stream_pick,
                    const uint64_t *rp, int64_t n_rows, uint64_t n, const uint8_t *smask, const int64_t *pool,
                    int64_t pool_size, double pb, uint32_t *col, int32_t threads) {
    if (threads < 1) threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    targets_job *jobs = (targets_job *)malloc(sizeof(targets_job) * (size_t)threads);
    const uint64_t E = rp[n_rows];
    int64_t r = 0;
    for (int32_t t = 0; t < threads; ++t) {
        /* split by edges so heavy rows spread over threads */
        uint64_t target = E * (uint64_t)(t + 1) / (uint64_t)threads;
        int64_t r1 = r;
        while (r1 < n_rows && rp[r1] < target) ++r1;
        if (t == threads - 1) r1 = n_rows;
        jobs[t] = (targets_job){rp, r, r1, n, stream_key(seed, stream_tgt), stream_key(seed, stream_bias),
                                stream_key(seed, stream_pick), smask, pool, pool_size, pb, col, 0};
        r = r1;
        pthread_create(&th[t], NULL, targets_worker, &jobs[t]);
    }
    int64_t failed = 0;
    for (int32_t t = 0; t < threads; ++t) {
        pthread_join(th[t], NULL);
        failed |= jobs[t].failed;
    }
    free(th);
    free(jobs);
    return failed ? -1 : 0;
}

/* Stable transpose of a CSR: inverse rows list their subjects ascending. */
void fastgen_transpose(const uint64_t *rp, const uint32_t *col, int64_t n, uint64_t *irp, uint32_t *icol) {
    memset(irp, 0, sizeof(uint64_t) * (size_t)(n + 1));
    const uint64_t E = rp[n];
    for (uint64_t k = 0; k < E; ++k) irp[col[k] + 1] += 1;
    for (int64_t i = 0; i < n; ++i) irp[i + 1] += irp[i];
    uint64_t *cur = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    memcpy(cur, irp, sizeof(uint64_t) * (size_t)n);
    for (int64_t a = 0; a < n; ++a)
        for (uint64_t k = rp[a]; k < rp[a + 1]; ++k) icol[cur[col[k]]++] = (uint32_t)a;
    free(cur);
}

typedef struct {
    uint64_t key;
    double p_in, p_out;
    const uint8_t *z;
    uint64_t i0, i1;
    uint8_t *out;   /* packed little-endian bits */
} bern_job;

static void *bern_worker(void *arg) {
    bern_job *j = (bern_job *)arg;
    for (uint64_t i = j->i0; i < j->i1; i += 8) {
        uint8_t b = 0;
        for (int q = 0; q < 8; ++q) {
            uint64_t k = i + (uint64_t)q;
            if (k >= j->i1) break;
            double p = (j->z && j->z[k]) ? j->p_in : j->p_out;
            if (uniform(j->key, k) < p) b |= (uint8_t)(1u << q);
        }
        j->out[i >> 3] = b;
    }
    return NULL;
}

/* Bernoulli membership bits of one concept: bit i set iff uniform(i) < p
 * (p_in for individuals with z[i] != 0 when z is given, else p_out). */
void fastgen_bernoulli(uint64_t seed, uint64_t stream, uint64_t n, double p_out, double p_in, const uint8_t *z,
                       uint8_t *out, int32_t threads) {
    if (threads < 1) threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    bern_job *jobs = (bern_job *)malloc(sizeof(bern_job) * (size_t)threads);
    uint64_t key = stream_key(seed, stream);
    for (int32_t t = 0; t < threads; ++t) {
        uint64_t i0 = (n * (uint64_t)t / (uint64_t)threads) & ~7ull;
        uint64_t i1 = t == threads - 1 ? n : ((n * (uint64_t)(t + 1) / (uint64_t)threads) & ~7ull);
        jobs[t] = (bern_job){key, p_in, p_out, z, i0, i1, out};
        pthread_create(&th[t], NULL, bern_worker, &jobs[t]);
    }
    for (int32_t t = 0; t < threads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
}

/* ------------------------------------------------------------------ refinements
 * The refinement generator of synth/refine.py (Refiner.refine) on postfix
 * programs, draw for draw: candidate k refines beam member k mod n_beam with
 * the sequential stream (seed, S_REFINE + (step << 40) + (member << 24) + k).
 * Op codes and the instruction layout are those of synth/programs.py. */
enum { R_ATOM = 1, R_AND = 5, R_OR = 6, R_EXISTS = 7, R_FORALL = 8, R_ATLEAST = 9, R_DGE = 12, R_DLE = 13 };
#define S_REFINE (11ull << 16)

typedef struct {
    uint64_t key, k;
} seq_rng;

static inline uint64_t seq_next(seq_rng *r) {
    r->k += 1;
    return mix64(r->key + r->k * GOLDEN);
}
static inline double seq_random(seq_rng *r) { return (double)(seq_next(r) >> 11) * (1.0 / 9007199254740992.0); }
static inline int64_t seq_randint(seq_rng *r, int64_t lo, int64_t hi) {   /* inclusive */
    uint64_t span = (uint64_t)(hi - lo + 1);
    return lo + (int64_t)(((seq_next(r) >> 32) * span) >> 32);
}
static inline uint64_t mk(uint32_t op, uint32_t flags, uint32_t a, uint32_t b) {
    return (uint64_t)(op & 0xFF) | ((uint64_t)(flags & 0xFF) << 8) | ((uint64_t)(a & 0xFFFF) << 16) |
           ((uint64_t)b << 32);
}
static inline uint32_t f32bits(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    return u;
}
static inline float bitsf32(uint32_t u) {
    float x;
    memcpy(&x, &u, 4);
    return x;
}

/* a simple operand: atom (1/2), grid data restriction (3/10) or (some r A) (1/5) */
static int64_t simple(seq_rng *r, int64_t nc, int64_t nr, int64_t np_, const float *grid, const int64_t *goff,
                      uint64_t *out) {
    double u = seq_random(r);
    if (u < 0.5 || (np_ == 0 && nr == 0)) {
        out[0] = mk(R_ATOM, 0, (uint32_t)seq_randint(r, 0, nc - 1), 0);
        return 1;
    }
    if ((u < 0.8 && np_) || !nr) {
        int64_t p = seq_randint(r, 0, np_ - 1);
        int64_t gl = goff[p + 1] - goff[p];
        float t = grid[goff[p] + seq_randint(r, 0, gl - 1)];
        uint32_t op = seq_random(r) < 0.5 ? R_DGE : R_DLE;
        out[0] = mk(op, 0, (uint32_t)p, f32bits(t));
        return 1;
    }
    int64_t role = seq_randint(r, 0, nr - 1);
    uint32_t inv = seq_random(r) < 0.5 ? 1u : 0u;
    out[0] = mk(R_ATOM, 0, (uint32_t)seq_randint(r, 0, nc - 1), 0);
    out[1] = mk(R_EXISTS, inv, (uint32_t)role, 0);
    return 2;
}

/* Writes count candidates into out (capacity cap instructions) and their
 * offsets into out_offs[count+1]; returns 0, or -1 if cap is too small. */
int fastgen_refine(uint64_t seed, uint64_t step, const uint64_t *beam, const int64_t *boffs, int64_t n_beam,
                   int64_t count, int64_t nc, int64_t nr, int64_t np_, const float *grid, const int64_t *goff,
                   uint64_t *out, int64_t cap, int64_t *out_offs) {
    int64_t o = 0;
    out_offs[0] = 0;
    for (int64_t k = 0; k < count; ++k) {
        const int64_t m = k % n_beam;
        const uint64_t *base = beam + boffs[m];
        const int64_t bl = boffs[m + 1] - boffs[m];
        if (o + bl + 3 > cap) return -1;
        seq_rng r = {stream_key(seed, S_REFINE + (step << 40) + ((uint64_t)m << 24) + (uint64_t)k), 0};
        uint64_t *dst = out + o;
        memcpy(dst, base, sizeof(uint64_t) * (size_t)bl);
        int64_t len = bl;
        int64_t op = seq_randint(&r, 0, 3);
        int done = 0;
        if (op == 3) {
            int64_t nd = 0;
            for (int64_t i = 0; i < bl; ++i) {
                uint32_t c = (uint32_t)(base[i] & 0xFF);
                if (c == R_DGE || c == R_DLE) ++nd;
            }
            if (nd) {
                int64_t pick = seq_randint(&r, 0, nd - 1), at = -1;
                for (int64_t i = 0, seen = 0; i < bl; ++i) {
                    uint32_t c = (uint32_t)(base[i] & 0xFF);
                    if (c == R_DGE || c == R_DLE) {
                        if (seen == pick) {
                            at = i;
                            break;
                        }
                        ++seen;
                    }
                }
                const uint32_t c = (uint32_t)(base[at] & 0xFF), p = (uint32_t)((base[at] >> 16) & 0xFFFF);
                const float t = bitsf32((uint32_t)(base[at] >> 32));
                const float *g = grid + goff[p];
                const int64_t gl = goff[p + 1] - goff[p];
                int64_t i = 0;   /* first index with g[i] >= t (numpy searchsorted, NaN sorts last) */
                if (t != t) i = gl;
                else
                    while (i < gl && g[i] < t) ++i;
                int64_t j = c == R_DGE ? ((i < gl && g[i] == t) ? i + 1 : i) : i - 1;
                if (j >= 0 && j < gl) {
                    dst[at] = mk(c, 0, p, f32bits(g[j]));
                    done = 1;
                }
            }
            if (!done) op = 0;
        }
        if (!done) {
            if (op == 0 || op == 1) {
                len += simple(&r, nc, nr, np_, grid, goff, dst + len);
                dst[len++] = mk(op == 0 ? R_AND : R_OR, 0, 0, 0);
            } else {
                int64_t w = seq_randint(&r, 0, 2);
                int64_t role = nr ? seq_randint(&r, 0, nr - 1) : 0;
                uint32_t inv = seq_random(&r) < 0.5 ? 1u : 0u;
                if (w == 0 || !nr) {
                    if (nr) dst[len++] = mk(R_EXISTS, inv, (uint32_t)role, 0);
                    else {
                        len += simple(&r, nc, nr, np_, grid, goff, dst + len);
                        dst[len++] = mk(R_AND, 0, 0, 0);
                    }
                } else if (w == 1) {
                    dst[len++] = mk(R_FORALL, inv, (uint32_t)role, 0);
                } else {
                    dst[len++] = mk(R_ATLEAST, inv, (uint32_t)role, (uint32_t)seq_randint(&r, 1, 4));
                }
            }
        }
        o += len;
        out_offs[k + 1] = o;
    }
    return 0;
}
