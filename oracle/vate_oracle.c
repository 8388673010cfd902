/*
 * vate_oracle.c -- plain, slow, obviously-correct CPU oracle for VATE
 * (virtual asynchronous timestamp estimator, arXiv 1812.00282).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this
 * file: only the tests, the smoke check and the CPU-baseline leg of the bench
 * use it.  It shares no code, header or constant table with the CUDA library.
 *
 * Everything here follows the paper step by step, one AT and one pair at a
 * time, in double precision where floating point is involved:
 *   - AT value domain [0, 2k], 2k = inactive; InitAT / SetAT      (Sec. 3)
 *   - ACT recurrence                                               (Eq. 3)
 *   - CheckAT                                                      (Algorithm 1)
 *   - PreserveAT, general form                                     (Algorithm 2)
 *   - PreserveAT, fast form used on ACT in {0, k}                  (Algorithm 3, Corollary 1)
 *   - AT pool split into 2k blocks, BACT of block i               (Eq. 6-8)
 *   - block sizes a, b and the map AT -> block                     (Eq. 9-10)
 *   - low-deviation partition a', b'                               (Sec. 4.1, Fig. "low deviation partition")
 *   - virtual AT vector VAT_i = ATP[H(aip, i)], vid = BH(bip)      (Sec. 4.1)
 *   - estimator g*ln(Z_p) - g*ln(Z_v)  (sign reading, see below)   (Eq. 11, Eq. 2, Eq. 1)
 *   - per-slice loop: scan, estimate, BACT0+1, preserve 2 blocks  (Algorithm 4)
 *   - DR counters (VDRE) as an independent cross-check             (Sec. 1, Sec. 5)
 *
 * Readings where the paper is silent or inconsistent:
 *   R1  Eq. 11 / Eq. 2 are printed as g ln Z_v - g ln Z_p, which is <= 0 in
 *       normal use; the oracle evaluates g ln Z_p - g ln Z_v, the form that
 *       reduces to the linear estimator of Eq. 1 when Z_p = 1.
 *   R2  Algorithm 4 writes a = 2^c / k for the block size; Eq. 9 writes
 *       a = 2^c / (2k-1).  Eq. 9-10 (integer floor) is used; block(pid) = pid / a.
 *   R3  Algorithm 4 calls SetAT inside the maintenance loop; the prose of
 *       Sec. 4.1/4.2 says the blocks are maintained (PreserveAT); PreserveAT
 *       (Algorithm 3) is used.
 *   R5  Algorithm 3 is normative; Algorithm 2 is kept as a cross-check (they
 *       differ only when Value == ACT at a maintenance point, a state no run
 *       from InitAT can reach).
 *   R7  H and BH are "random hash functions" in the paper; the oracle fixes
 *       them to published mixers: BH is the SplitMix64 output function
 *       (Steele, Lea & Flood 2014) with Lemire's multiply-shift range
 *       reduction; H places the g virtual ATs of a host in segments of L
 *       consecutive pool ATs, segment j at the top bits of MurmurHash3's
 *       32-bit finalizer (Appleby) of the host's SplitMix64 key mixed with j.
 *   R10 saturation: V0 = g - A == 0 is replaced by 1 (flag SAT); a pool
 *       census with N0 == 0 is replaced by 1 (flag POOLFULL).
 *
 * Threads: the loops over pool ATs (census, inactive count) and over hosts
 * (estimate, per-age counts) may run on several OpenMP threads -- plain
 * parallel loops, no blocking or reordering of any per-AT or per-host step;
 * the integer sums do not depend on the split, so the results are the same
 * for any thread count.  The default is one thread (vo_set_threads).
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC -o liboracle.so vate_oracle.c -lm
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <omp.h>

/* Number of threads of the parallel loops below (1 by default). */
static int vo_nthreads = 1;
void vo_set_threads(int n) { vo_nthreads = n < 1 ? 1 : n; }
int vo_get_threads(void) { return vo_nthreads; }

/* ------------------------------------------------------------------ */
/* Hash functions H and BH (reading R7).                               */
/* ------------------------------------------------------------------ */

/* SplitMix64 output function: add the golden gamma, then two
 * xor-shift-multiply rounds and a final xor-shift. */
uint64_t vo_mix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* MurmurHash3's 32-bit finalizer (fmix32, Appleby): xor-shift-multiply
 * twice and a final xor-shift; a bijection on 32-bit words. */
uint32_t vo_fmix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x85EBCA6BU;
    x ^= x >> 13;
    x *= 0xC2B2AE35U;
    x ^= x >> 16;
    return x;
}

typedef struct {
    /* parameters (Algorithm 4 "Require": c, k; Sec. 4.1: g) */
    uint32_t c;          /* pool holds P = 2^c ATs                          */
    uint32_t k;          /* longest window, in slices                       */
    uint32_t g;          /* virtual ATs per host                            */
    uint32_t L;          /* segment length of the VAT placement (R7)        */
    uint32_t partition;  /* 0: Eq. 9-10; 1: low-deviation partition         */
    uint64_t seed;
    /* derived */
    uint64_t P;
    uint64_t key_h, key_bh;
    uint64_t a, b;       /* Eq. 9-10 (partition 0) or a', b' (partition 1)  */
    /* state */
    uint16_t *pool;      /* ATP: one AT value per element (values <= 2k)    */
    uint32_t bact0;      /* BACT^0 (Eq. 7)                                  */
    int64_t  t;          /* current slice number, origin 0                  */
    /* VDRE cross-check: one DR per pool position (Sec. 1, Sec. 5) */
    uint16_t *dr;
} vo_state;

/* BH(bip) in [0, g): high 32 bits of the mix, scaled by g (Lemire). */
uint32_t vo_bh(const vo_state *s, uint32_t bip)
{
    uint64_t m = vo_mix64(s->key_bh ^ (uint64_t)bip);
    uint64_t hi = m >> 32;
    return (uint32_t)((hi * (uint64_t)s->g) >> 32);
}

/* H(aip, i) in [0, P): the i-th virtual AT of host aip.  With segment
 * length L, VAT i lives at offset (i mod L) inside pool segment
 * seg(aip, j), j = floor(i / L).  The host's key is the 64-bit mix
 * K = mix64(key_h ^ aip << 32); seg(aip, j) is the top (c - log2 L) bits of
 * fmix32(low32(K) ^ j * 0x9E3779B9) ^ high32(K). */
uint64_t vo_h(const vo_state *s, uint32_t aip, uint32_t i)
{
    uint32_t log2L = 0;
    while ((1u << log2L) < s->L) log2L++;
    uint32_t j = i / s->L;
    uint32_t o = i % s->L;
    uint32_t segbits = s->c - log2L;
    uint64_t K = vo_mix64(s->key_h ^ (((uint64_t)aip) << 32));
    uint32_t x = vo_fmix32((uint32_t)K ^ (uint32_t)(j * 0x9E3779B9U)) ^ (uint32_t)(K >> 32);
    uint64_t seg = (uint64_t)x >> (32 - segbits);
    return seg * (uint64_t)s->L + (uint64_t)o;
}

/* The same H and BH without a pool, for pools too large to hold here: a
 * state with only the hash parameters filled in. */
uint64_t vo_h_of(uint32_t c, uint32_t L, uint64_t seed, uint32_t aip, uint32_t i)
{
    vo_state s;
    memset(&s, 0, sizeof s);
    s.c = c;
    s.L = L;
    s.key_h = vo_mix64(seed + 1);
    return vo_h(&s, aip, i);
}

uint32_t vo_bh_of(uint32_t g, uint64_t seed, uint32_t bip)
{
    vo_state s;
    memset(&s, 0, sizeof s);
    s.g = g;
    s.key_bh = vo_mix64(seed + 2);
    return vo_bh(&s, bip);
}

/* ------------------------------------------------------------------ */
/* AT blocks (Eq. 6-10).                                               */
/* ------------------------------------------------------------------ */

/* Block index of pool AT number pid. */
uint32_t vo_block(const vo_state *s, uint64_t pid)
{
    if (s->partition == 0) {
        /* Eq. 9-10: blocks 0..2k-2 hold a ATs each, block 2k-1 holds b. */
        return (uint32_t)(pid / s->a);
    }
    /* Low-deviation partition: the first 2k-b' blocks hold a' ATs, the
     * last b' blocks hold a'+1 ATs (Sec. 4.1). */
    uint64_t twok = 2ull * s->k;
    uint64_t first = s->a * (twok - s->b);
    if (pid < first) return (uint32_t)(pid / s->a);
    return (uint32_t)((pid + twok - s->b) / (s->a + 1));
}

/* First pool AT of block i and the number of ATs in it. */
void vo_block_range(const vo_state *s, uint32_t i, uint64_t *start, uint64_t *count)
{
    uint64_t twok = 2ull * s->k;
    if (s->partition == 0) {
        *start = (uint64_t)i * s->a;
        *count = (i + 1 < twok) ? s->a : s->b;
        return;
    }
    uint64_t nsmall = twok - s->b;
    if (i < nsmall) { *start = (uint64_t)i * s->a; *count = s->a; }
    else { *start = nsmall * s->a + (uint64_t)(i - nsmall) * (s->a + 1); *count = s->a + 1; }
}

/* ACT of block i in the current slice: (BACT^0 + i) mod 2k (Eq. 8). */
uint32_t vo_bact(const vo_state *s, uint32_t i)
{
    return (s->bact0 + i) % (2 * s->k);
}

/* ACT of the AT at pool position pid. */
uint32_t vo_act_of(const vo_state *s, uint64_t pid)
{
    return vo_bact(s, vo_block(s, pid));
}

/* ------------------------------------------------------------------ */
/* The four AT operations (Sec. 3).                                    */
/* ------------------------------------------------------------------ */

/* Algorithm 1: is an AT with value v active in W(t-k'+1, k') when its
 * ACT is act?  Value 2k means inactive. */
int vo_check_at(uint32_t v, uint32_t act, uint32_t k, uint32_t kprime)
{
    if (v == 2 * k) return 0;
    uint32_t dis = (act + 2 * k - v) % (2 * k);
    return dis <= kprime - 1;
}

/* Algorithm 2: general PreserveAT -- mark inactive when the distance is k or more. */
uint32_t vo_preserve_general(uint32_t v, uint32_t act, uint32_t k)
{
    if (v == 2 * k) return v;
    uint32_t dis = (act + 2 * k - v) % (2 * k);
    if (dis >= k) return 2 * k;
    return v;
}

/* Algorithm 3: fast PreserveAT, only meaningful when act is 0 or k
 * (Corollary 1).  At act = 0 values 0..k expire; at act = k values
 * k..2k-1 and 0 expire. */
uint32_t vo_preserve_fast(uint32_t v, uint32_t act, uint32_t k)
{
    if (act == 0) {
        if (v <= k) return 2 * k;
    }
    if (act == k) {
        if (v >= k && v <= 2 * k - 1) return 2 * k;
        if (v == 0) return 2 * k;
    }
    return v;
}

/* ------------------------------------------------------------------ */
/* State life cycle (Algorithm 4).                                     */
/* ------------------------------------------------------------------ */

/* Returns NULL when the parameters are outside what the method allows:
 * every block index must stay below 2k (so a >= b), L must be a power of two
 * dividing g, and c - log2 L must leave at least one segment bit. */
vo_state *vo_create(uint32_t c, uint32_t k, uint32_t g, uint32_t L,
                    uint32_t partition, uint64_t seed)
{
    if (c < 1 || c > 32 || k < 1 || k > 1023 || g < 1 || L < 1) return NULL;
    if ((L & (L - 1)) != 0 || g % L != 0 || partition > 1) return NULL;
    uint32_t log2L = 0;
    while ((1u << log2L) < L) log2L++;
    if (c <= log2L) return NULL;
    uint64_t P = 1ull << c;
    uint64_t twok = 2ull * k;
    if (P < (twok - 1) * twok) return NULL;

    vo_state *s = (vo_state *)calloc(1, sizeof(vo_state));
    if (!s) return NULL;
    s->c = c; s->k = k; s->g = g; s->L = L; s->partition = partition; s->seed = seed;
    s->P = P;
    s->key_h = vo_mix64(seed + 1);
    s->key_bh = vo_mix64(seed + 2);
    if (partition == 0) {          /* Eq. 9 and Eq. 10 */
        s->a = P / (twok - 1);
        s->b = P % (twok - 1);
    } else {                       /* low-deviation partition */
        s->a = P / twok;
        s->b = P % twok;
    }
    s->pool = (uint16_t *)malloc(P * sizeof(uint16_t));
    s->dr = (uint16_t *)malloc(P * sizeof(uint16_t));
    if (!s->pool || !s->dr) { free(s->pool); free(s->dr); free(s); return NULL; }
    /* InitAT on every AT of the pool; BACT^0 = 0; t = 0. */
    for (uint64_t i = 0; i < P; i++) s->pool[i] = (uint16_t)(2 * k);
    /* DR counters start "all ones", i.e. inactive; k or more is inactive. */
    for (uint64_t i = 0; i < P; i++) s->dr[i] = (uint16_t)k;
    s->bact0 = 0;
    s->t = 0;
    return s;
}

void vo_destroy(vo_state *s)
{
    if (!s) return;
    free(s->pool);
    free(s->dr);
    free(s);
}

uint64_t vo_pool_size(const vo_state *s) { return s->P; }
uint32_t vo_bact0(const vo_state *s) { return s->bact0; }
int64_t vo_slice(const vo_state *s) { return s->t; }
uint64_t vo_block_a(const vo_state *s) { return s->a; }
uint64_t vo_block_b(const vo_state *s) { return s->b; }
void vo_copy_pool(const vo_state *s, uint16_t *dst) { memcpy(dst, s->pool, s->P * sizeof(uint16_t)); }
void vo_copy_dr(const vo_state *s, uint16_t *dst) { memcpy(dst, s->dr, s->P * sizeof(uint16_t)); }

/* SetAT on one pool AT: its value becomes the ACT of its block. */
void vo_set_pid(vo_state *s, uint64_t pid)
{
    s->pool[pid] = (uint16_t)vo_act_of(s, pid);
    s->dr[pid] = 0;   /* the DR of the same position records distance 0 */
}

/* SetAT on a list of pool ATs (tests that drive single ATs). */
void vo_set_pids(vo_state *s, const uint64_t *pids, uint64_t n)
{
    for (uint64_t q = 0; q < n; q++) vo_set_pid(s, pids[q]);
}

/* Scan of one slice's pairs, in stream order (Algorithm 4, scan loop):
 * vid = BH(bip); pid = H(aip, vid); bid = block(pid); act = (BACT0+bid) mod 2k;
 * SetAT(ATP[pid]).  pairs holds n (aip, bip) records, aip first. */
void vo_ingest(vo_state *s, const uint32_t *pairs, uint64_t n)
{
    for (uint64_t p = 0; p < n; p++) {
        uint32_t aip = pairs[2 * p];
        uint32_t bip = pairs[2 * p + 1];
        uint32_t vid = vo_bh(s, bip);
        uint64_t pid = vo_h(s, aip, vid);
        vo_set_pid(s, pid);
    }
}

/* Pool positions hit by each pair, for tests (same arithmetic as vo_ingest). */
void vo_pids_of_pairs(const vo_state *s, const uint32_t *pairs, uint64_t n, uint64_t *out)
{
    for (uint64_t p = 0; p < n; p++) {
        uint32_t vid = vo_bh(s, pairs[2 * p + 1]);
        out[p] = vo_h(s, pairs[2 * p], vid);
    }
}

/* End of the slice: slide the window and maintain the two blocks whose
 * ACT became 0 or k (Algorithm 4, last lines; Algorithm 3).  The DR pool
 * of the VDRE cross-check ages every counter by one (Sec. 1). */
void vo_advance(vo_state *s)
{
    uint32_t twok = 2 * s->k;
    s->bact0 = (s->bact0 + 1) % twok;
    s->t += 1;
    for (uint32_t i = 0; i < twok; i++) {
        uint32_t bact = vo_bact(s, i);
        if (bact == 0 || bact == s->k) {
            uint64_t start, count;
            vo_block_range(s, i, &start, &count);
            for (uint64_t q = start; q < start + count; q++)
                s->pool[q] = (uint16_t)vo_preserve_fast(s->pool[q], bact, s->k);
        }
    }
    for (uint64_t q = 0; q < s->P; q++)
        if (s->dr[q] < s->k) s->dr[q] += 1;
}

/* Same as vo_advance but maintaining every AT with Algorithm 2 (the general
 * form) in every slice, for the Algorithm 2 / Algorithm 3 cross-check. */
void vo_advance_general_every_slice(vo_state *s)
{
    uint32_t twok = 2 * s->k;
    s->bact0 = (s->bact0 + 1) % twok;
    s->t += 1;
    for (uint64_t q = 0; q < s->P; q++)
        s->pool[q] = (uint16_t)vo_preserve_general(s->pool[q], vo_act_of(s, q), s->k);
    for (uint64_t q = 0; q < s->P; q++)
        if (s->dr[q] < s->k) s->dr[q] += 1;
}

/* Active flag of every pool AT for window k' (Algorithm 1 on each AT). */
void vo_check_all(const vo_state *s, uint32_t kprime, uint8_t *out)
{
    for (uint64_t q = 0; q < s->P; q++)
        out[q] = (uint8_t)vo_check_at(s->pool[q], vo_act_of(s, q), s->k, kprime);
}

/* Pool census: hist[d] = number of pool ATs at distance d (0 <= d < 2k),
 * hist[2k] = number of inactive ATs (value 2k).  The distance is the
 * quantity Algorithm 1 compares with k'-1. */
void vo_census(const vo_state *s, uint64_t *hist)
{
    uint32_t twok = 2 * s->k;
    for (uint32_t d = 0; d <= twok; d++) hist[d] = 0;
#pragma omp parallel for num_threads(vo_nthreads) reduction(+ : hist[:twok + 1]) schedule(static)
    for (uint64_t q = 0; q < s->P; q++) {
        uint32_t v = s->pool[q];
        if (v == twok) { hist[twok]++; continue; }
        uint32_t act = vo_act_of(s, q);
        hist[(act + twok - v) % twok]++;
    }
}

/* Number of pool ATs that are inactive in W(t-k'+1, k'): Z_p = N0 / P. */
uint64_t vo_pool_inactive(const vo_state *s, uint32_t kprime)
{
    uint64_t n0 = 0;
#pragma omp parallel for num_threads(vo_nthreads) reduction(+ : n0) schedule(static)
    for (uint64_t q = 0; q < s->P; q++)
        if (!vo_check_at(s->pool[q], vo_act_of(s, q), s->k, kprime)) n0++;
    return n0;
}

/* Inactive ATs for window k' among pool positions [start, end) (a bounded
 * sample of the census, for timing on a slice of the pool). */
uint64_t vo_pool_inactive_range(const vo_state *s, uint32_t kprime, uint64_t start, uint64_t end)
{
    uint64_t n0 = 0;
    if (end > s->P) end = s->P;
#pragma omp parallel for num_threads(vo_nthreads) reduction(+ : n0) schedule(static)
    for (uint64_t q = start; q < end; q++)
        if (!vo_check_at(s->pool[q], vo_act_of(s, q), s->k, kprime)) n0++;
    return n0;
}

/* Eq. 11 for one host, given the host's active VAT count A (out of g)
 * and the pool's inactive count N0 (out of P).  Reading R1 for the sign,
 * R10 for the two degenerate cases.  flags bit 0 = SAT, bit 1 = POOLFULL. */
double vo_estimate_from_counts(uint32_t g, uint64_t P, uint64_t N0, uint32_t A, uint8_t *flags)
{
    uint8_t f = 0;
    uint64_t V0 = (uint64_t)g - A;
    if (V0 == 0) { V0 = 1; f |= 1; }
    if (N0 == 0) { N0 = 1; f |= 2; }
    double Zv = (double)V0 / (double)g;
    double Zp = (double)N0 / (double)P;
    if (flags) *flags = f;
    return (double)g * log(Zp) - (double)g * log(Zv);
}

/* Active VAT count of one host: A = #{ i < g : CheckAT(ATP[H(aip,i)], k') }. */
uint32_t vo_active_vats(const vo_state *s, uint32_t aip, uint32_t kprime)
{
    uint32_t A = 0;
    for (uint32_t i = 0; i < s->g; i++) {
        uint64_t pid = vo_h(s, aip, i);
        A += (uint32_t)vo_check_at(s->pool[pid], vo_act_of(s, pid), s->k, kprime);
    }
    return A;
}

/* Estimation step of Algorithm 4 for a list of hosts: Z_p from the pool,
 * Z_v from each host's g VATs, then Eq. 11.  Any of the outputs may be NULL. */
void vo_estimate_hosts(const vo_state *s, const uint32_t *aips, uint64_t n, uint32_t kprime, uint64_t N0,
                       double *est, uint32_t *active, uint8_t *flags);

void vo_estimate(const vo_state *s, const uint32_t *aips, uint64_t n, uint32_t kprime,
                 double *est, uint32_t *active, uint8_t *flags)
{
    vo_estimate_hosts(s, aips, n, kprime, vo_pool_inactive(s, kprime), est, active, flags);
}

/* The per-host part of the estimation step, given the pool's inactive count
 * N0 for window k' (Z_p = N0 / P). */
void vo_estimate_hosts(const vo_state *s, const uint32_t *aips, uint64_t n, uint32_t kprime, uint64_t N0,
                       double *est, uint32_t *active, uint8_t *flags)
{
#pragma omp parallel for num_threads(vo_nthreads) schedule(dynamic, 16)
    for (uint64_t h = 0; h < n; h++) {
        uint32_t A = vo_active_vats(s, aips[h], kprime);
        uint8_t f = 0;
        double e = vo_estimate_from_counts(s->g, s->P, N0, A, &f);
        if (est) est[h] = e;
        if (active) active[h] = A;
        if (flags) flags[h] = f;
    }
}

/* Per-age VAT counts of each host: out[h*k + d] = number of the host's g
 * VATs whose distance is exactly d (0 <= d < k), i.e. ATs last set d slices
 * ago.  The active count for window k' is the sum of the first k' entries. */
void vo_age_counts(const vo_state *s, const uint32_t *aips, uint64_t n, uint32_t *out)
{
    uint32_t twok = 2 * s->k;
#pragma omp parallel for num_threads(vo_nthreads) schedule(dynamic, 16)
    for (uint64_t h = 0; h < n; h++) {
        uint32_t *row = out + h * s->k;
        for (uint32_t d = 0; d < s->k; d++) row[d] = 0;
        for (uint32_t i = 0; i < s->g; i++) {
            uint64_t pid = vo_h(s, aips[h], i);
            uint32_t v = s->pool[pid];
            if (v == twok) continue;
            uint32_t d = (vo_act_of(s, pid) + twok - v) % twok;
            if (d < s->k) row[d]++;
        }
    }
}

/* VDRE cross-check: active VAT count from the DR pool (a DR below k' is
 * active in W(t-k'+1, k'), Sec. 1). */
uint32_t vo_active_vats_dr(const vo_state *s, uint32_t aip, uint32_t kprime)
{
    uint32_t A = 0;
    for (uint32_t i = 0; i < s->g; i++)
        A += (uint32_t)(s->dr[vo_h(s, aip, i)] < kprime);
    return A;
}

/* Overwrite the pool (tests that construct states by hand). */
void vo_load_pool(vo_state *s, const uint16_t *src) { memcpy(s->pool, src, s->P * sizeof(uint16_t)); }
