/*
 * nsgen.c -- seeded synthetic packet-stream generators.
 *
 * This module only draws inputs: anonymized (src, dst) uint32 address pairs
 * shaped like the network-sensing challenge's packet windows (2^30 packets in
 * total, 2^17 per window, 32-bit anonymized addresses; paper, section "Graph
 * Challenge Setup", paragraph "Inputs", and section "Implementation",
 * paragraph "IP Address Anonymization").  It holds none of the traffic-matrix
 * arithmetic; both the CPU oracle and the CUDA library consume its output.
 *
 * Every draw is counter-based, so the bytes do not depend on the thread count:
 *   rand64(seed, stream, i) = splitmix64(seed ^ (stream << 40) ^ i)
 * where splitmix64 is Steele, Lea and Flood's SplitMix64 output function
 * ("Fast splittable pseudorandom number generators", OOPSLA 2014), applied
 * to its argument plus the golden-ratio increment.
 *
 * Address relabelling uses a keyed 4-round Feistel network on 16-bit halves,
 * a bijection on [0, 2^32) by construction (Luby-Rackoff structure).
 *
 * Zipf(s) over ranks 1..K uses rejection-inversion against the continuous
 * hat x^-s on [1/2, K+1/2] (Hoermann and Derflinger, ACM TOMACS 1996):
 * because x^-s is convex, the hat mass of the cell [k-1/2, k+1/2] is at least
 * k^-s, so drawing X from the hat, rounding it to k, and keeping k when the
 * inverted uniform lies in the top k^-s of that cell's mass samples exactly
 * P(k) proportional to k^-s.
 *
 * RMAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): each of `scale` levels picks
 * a quadrant with probabilities (a, b, c, d); the quadrant bits form src (c,d)
 * and dst (b,d) from the most significant bit down.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define NSG_GOLDEN 0x9E3779B97F4A7C15ull

uint64_t nsg_splitmix64(uint64_t x) {
    uint64_t z = x + NSG_GOLDEN;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t nsg_rand64(uint64_t seed, uint64_t stream, uint64_t i) {
    return nsg_splitmix64(seed ^ (stream << 40) ^ i);
}

/* out[i] = nsg_rand64(seed, stream, i): random 64-bit keys, e.g. the ones an
 * anonymizing permutation is drawn from */
void nsg_rand64_fill(uint64_t* out, uint64_t n, uint64_t seed, uint64_t stream) {
    for (uint64_t i = 0; i < n; ++i) out[i] = nsg_rand64(seed, stream, i);
}

/* uniform double in [0, 1) with 53 random bits */
static inline double u01(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }

/* ---- keyed Feistel bijection on 32 bits -------------------------------- */

static inline uint32_t feistel_f(uint32_t half, uint64_t key, int round) {
    uint64_t z = nsg_splitmix64(key ^ ((uint64_t)round << 56) ^ (uint64_t)half);
    return (uint32_t)(z & 0xFFFFu);
}

uint32_t nsg_feistel(uint32_t x, uint64_t key) {
    uint32_t l = x >> 16, r = x & 0xFFFFu;
    for (int k = 0; k < 4; ++k) {
        uint32_t nl = r;
        uint32_t nr = l ^ feistel_f(r, key, k);
        l = nl;
        r = nr;
    }
    return (l << 16) | r;
}

uint32_t nsg_feistel_inv(uint32_t y, uint64_t key) {
    uint32_t l = y >> 16, r = y & 0xFFFFu;
    for (int k = 3; k >= 0; --k) {
        uint32_t pr = l;
        uint32_t pl = r ^ feistel_f(l, key, k);
        l = pl;
        r = pr;
    }
    return (l << 16) | r;
}

void nsg_feistel_fill(const uint32_t* in, uint32_t* out, uint64_t n, uint64_t key) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = nsg_feistel(in[i], key);
}

/* ---- Zipf by rejection-inversion ---------------------------------------- */

typedef struct {
    double s, one_minus_s, h_lo, h_hi;
    uint64_t K;
} zipf_t;

/* antiderivative of x^-s: (x^(1-s) - 1)/(1-s), or log x when s == 1 */
static inline double zH(const zipf_t* z, double x) {
    double lx = log(x);
    if (fabs(z->one_minus_s) < 1e-12) return lx;
    return expm1(z->one_minus_s * lx) / z->one_minus_s;
}
static inline double zHinv(const zipf_t* z, double y) {
    if (fabs(z->one_minus_s) < 1e-12) return exp(y);
    return exp(log1p(z->one_minus_s * y) / z->one_minus_s);
}
static void zipf_init(zipf_t* z, double s, uint64_t K) {
    z->s = s;
    z->one_minus_s = 1.0 - s;
    z->K = K;
    z->h_lo = zH(z, 0.5);
    z->h_hi = zH(z, (double)K + 0.5);
}
/* returns a rank in [0, K) (rank 0 is the most frequent) */
static inline uint64_t zipf_draw(const zipf_t* z, uint64_t seed, uint64_t stream, uint64_t i) {
    for (uint64_t attempt = 0;; ++attempt) {
        double u = u01(nsg_rand64(seed, stream + (attempt << 8), i));
        double y = z->h_hi + u * (z->h_lo - z->h_hi); /* in (h_lo, h_hi] */
        double x = zHinv(z, y);
        double kf = floor(x + 0.5);
        if (kf < 1.0) kf = 1.0;
        if (kf > (double)z->K) kf = (double)z->K;
        /* accept when y lies in the top k^-s of the cell [k-1/2, k+1/2] */
        double top = zH(z, kf + 0.5);
        double pk = exp(-z->s * log(kf));
        if (y >= top - pk) return (uint64_t)kf - 1;
        if (attempt > 1000) return (uint64_t)kf - 1; /* never reached in practice */
    }
}

/* One column (src or dst) of Zipf(s)-distributed ranks over K addresses,
 * relabelled into 32 bits by the keyed Feistel bijection. */
void nsg_zipf_fill(uint32_t* out, uint64_t n, double s, uint64_t K, uint64_t seed,
                   uint64_t stream, uint64_t bij_key) {
    zipf_t z;
    zipf_init(&z, s, K);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint64_t r = zipf_draw(&z, seed, stream, (uint64_t)i);
        out[i] = nsg_feistel((uint32_t)r, bij_key);
    }
}

/* Zipf ranks only (no relabelling), for distribution tests. */
void nsg_zipf_ranks(uint32_t* out, uint64_t n, double s, uint64_t K, uint64_t seed, uint64_t stream) {
    zipf_t z;
    zipf_init(&z, s, K);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = (uint32_t)zipf_draw(&z, seed, stream, (uint64_t)i);
}

/* ---- RMAT with uniform background --------------------------------------- */

/* Packet i of an RMAT stream of `scale` levels with quadrant probabilities
 * (a, b, c, 1-a-b-c); with probability bg_frac the pair is instead uniform
 * over 32 bits.  Both ends are then relabelled by the same bijection (one
 * anonymizing map for all addresses).  Packet indices start at i0 so that a
 * window can be drawn on its own. */
void nsg_rmat_fill(uint32_t* src, uint32_t* dst, uint64_t n, uint64_t i0, int scale, double a,
                   double b, double c, double bg_frac, uint64_t seed, uint64_t bij_key) {
    const double ta = a * 4294967296.0, tb = (a + b) * 4294967296.0,
                 tc = (a + b + c) * 4294967296.0, tbg = bg_frac * 4294967296.0;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < (int64_t)n; ++j) {
        uint64_t i = i0 + (uint64_t)j;
        uint64_t h = nsg_rand64(seed, 1, i);
        uint32_t s = 0, d = 0;
        if ((double)(uint32_t)h < tbg) {
            uint64_t w = nsg_rand64(seed, 2, i);
            s = (uint32_t)(w >> 32);
            d = (uint32_t)w;
        } else {
            uint64_t w = 0;
            for (int lev = 0; lev < scale; ++lev) {
                if ((lev & 1) == 0) w = nsg_rand64(seed, 16 + (uint64_t)(lev >> 1), i);
                uint32_t u = (lev & 1) ? (uint32_t)(w >> 32) : (uint32_t)w;
                double du = (double)u;
                uint32_t sb = du >= tb;              /* quadrants c, d: lower half */
                uint32_t db = (du >= ta && du < tb) || du >= tc; /* quadrants b, d */
                s = (s << 1) | sb;
                d = (d << 1) | db;
            }
        }
        src[j] = nsg_feistel(s, bij_key);
        dst[j] = nsg_feistel(d, bij_key);
    }
}

/* Window sizes log-uniform in [2^lo, 2^hi]: round(2^(lo + (hi-lo) u)). */
void nsg_loguniform_sizes(uint64_t* out, uint64_t k, double lo, double hi, uint64_t seed,
                          uint64_t stream) {
    for (uint64_t i = 0; i < k; ++i) {
        double u = u01(nsg_rand64(seed, stream, i));
        out[i] = (uint64_t)llround(exp2(lo + (hi - lo) * u));
    }
}

/* Uniform doubles in [lo, hi). */
void nsg_uniform_doubles(double* out, uint64_t k, double lo, double hi, uint64_t seed,
                         uint64_t stream) {
    for (uint64_t i = 0; i < k; ++i) out[i] = lo + (hi - lo) * u01(nsg_rand64(seed, stream, i));
}

/* Poisson-process arrival times (seconds) at the given rate: cumulative sums
 * of exponential gaps -log(1-u)/rate. */
void nsg_poisson_arrivals(double* out, uint64_t k, double rate, uint64_t seed, uint64_t stream) {
    double t = 0.0;
    for (uint64_t i = 0; i < k; ++i) {
        double u = u01(nsg_rand64(seed, stream, i));
        t += -log1p(-u) / rate;
        out[i] = t;
    }
}

/* Uniform 32-bit pairs masked to `bits` low bits (tiny address spaces for
 * brute-force tests). */
void nsg_uniform_pairs(uint32_t* src, uint32_t* dst, uint64_t n, int bits, uint64_t seed) {
    uint32_t mask = bits >= 32 ? 0xFFFFFFFFu : ((1u << bits) - 1u);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint64_t w = nsg_rand64(seed, 3, (uint64_t)i);
        src[i] = (uint32_t)(w >> 32) & mask;
        dst[i] = (uint32_t)w & mask;
    }
}
