// Host-only check of the SWAR AT arithmetic in vate_device.cuh against the
// scalar forms of Algorithm 1 (CheckAT), Eq. 5 (distance) and Algorithm 3
// (fast PreserveAT): every k <= 63, every ACT, every k' <= k, every AT value
// 0..2k in every byte position, plus random mixed words; and the byte clamp
// for every byte value.  The frame-0 forms
// (values kept as value minus block index, mod 2k) are tied to the paper's
// through the per-block map.  Prints "OK".
#include <cstdio>
#include <cstdlib>
#include "vate_device.cuh"

using namespace vate;

static uint32_t rng_state = 12345u;
static uint32_t rnd() { rng_state = rng_state * 1664525u + 1013904223u; return rng_state >> 8; }

// packed_count_word<B> against a field-by-field count, for timestamps in
// frame 0 (ACT = BACT^0) and recorders: every field range [fa, fb), every
// BACT^0 and k' (sampled when k is large), words with every value in every
// field position (B <= 6) or random ones.
template <int B>
static bool check_packed(long &checked) {
    constexpr uint32_t PN = 32u / B, MF = (1u << B) - 1u;
    const uint32_t kmax = ((1u << B) - 1u) / 2u;              // 2k + 1 <= 2^B
    for (uint32_t k = 1; k <= kmax; k += (k < 12 ? 1u : 1u + kmax / 7u)) {
        const uint32_t twok = 2u * k;
        for (uint32_t dr = 0; dr < 2; dr++)
            for (uint32_t bact0 = 0; bact0 < twok; bact0 += (twok <= 40 ? 1u : 1u + twok / 13u))
                for (uint32_t kp = 1; kp <= k; kp += (k <= 20 ? 1u : 1u + k / 9u)) {
                    const PackedRange r = dr ? packed_range_dr(B, kp, twok) : packed_range_at(B, bact0, kp, twok);
                    const int nw = B <= 6 ? (int)(PN << B) : 96;
                    for (int t = 0; t < nw; t++) {
                        uint32_t v[32];
                        for (uint32_t f = 0; f < PN; f++) v[f] = rnd() & MF;
                        if (B <= 6) v[(uint32_t)t >> B] = (uint32_t)t & MF;   // every value in every position
                        uint32_t w = (uint32_t)((uint64_t)rnd() << (PN * B));   // random unused top bits
                        for (uint32_t f = 0; f < PN; f++) w |= v[f] << (f * B);
                        for (uint32_t fa = 0; fa <= PN; fa++)
                            for (uint32_t fb = fa; fb <= PN; fb++) {
                                uint32_t want = 0;
                                for (uint32_t f = fa; f < fb; f++)
                                    want += dr ? (v[f] < kp) : (v[f] < twok && check_at(v[f], bact0, kp, twok));
                                if (packed_count_word<B>(w, r, fa, fb) != want) {
                                    printf("FAIL packed B=%d k=%u dr=%u bact0=%u k'=%u fields [%u,%u) w=%08x\n", B, k,
                                           dr, bact0, kp, fa, fb, w);
                                    return false;
                                }
                                checked++;
                            }
                    }
                }
    }
    return true;
}

int main() {
    long checked = 0;
    if (!check_packed<4>(checked) || !check_packed<5>(checked) || !check_packed<6>(checked) ||
        !check_packed<7>(checked) || !check_packed<8>(checked) || !check_packed<9>(checked) ||
        !check_packed<10>(checked) || !check_packed<11>(checked))
        return 1;
    // swar_clamp: every byte value in every position, every top <= 126, the
    // other bytes random (so that a carry across bytes would show)
    for (uint32_t top = 0; top <= 126; top++)
        for (uint32_t x = 0; x < 256; x++)
            for (int pos = 0; pos < 4; pos++) {
                uint32_t v[4];
                for (int b = 0; b < 4; b++) v[b] = rnd() & 0xFFu;
                v[pos] = x;
                const uint32_t w = v[0] | v[1] << 8 | v[2] << 16 | v[3] << 24;
                const uint32_t r = swar_clamp(w, top);
                for (int b = 0; b < 4; b++)
                    if (((r >> (8 * b)) & 0xFFu) != (v[b] > top ? top : v[b])) {
                        printf("FAIL clamp top=%u v=%u\n", top, v[b]);
                        return 1;
                    }
                checked++;
            }
    for (uint32_t k = 1; k <= 63; k++) {
        uint32_t twok = 2 * k;
        uint32_t c2k = (128u - twok) * ONES;
        for (uint32_t act = 0; act < twok; act++) {
            for (uint32_t kp = 1; kp <= k; kp++) {
                RangeConsts rc = range_consts(act, kp, twok);
                for (int trial = 0; trial < 64 + (int)(twok + 1) * 4; trial++) {
                    uint32_t v[4];
                    for (int b = 0; b < 4; b++) v[b] = rnd() % (twok + 1);
                    if (trial < (int)(twok + 1) * 4) {          // every value in every position
                        for (int b = 0; b < 4; b++) v[b] = twok;
                        v[trial & 3] = (uint32_t)(trial >> 2);
                    }
                    uint32_t w = v[0] | v[1] << 8 | v[2] << 16 | v[3] << 24;
                    uint32_t m = swar_active(w, rc, c2k);
                    uint32_t bins = swar_bins(w, act, twok);
                    for (int b = 0; b < 4; b++) {
                        bool want = check_at(v[b], act, kp, twok);
                        bool got = (m >> (8 * b + 7)) & 1u;
                        if (want != got || (m >> (8 * b)) & 0x7Fu) {
                            printf("FAIL active k=%u act=%u k'=%u v=%u\n", k, act, kp, v[b]);
                            return 1;
                        }
                        uint32_t wantbin = v[b] == twok ? twok : (act + twok - v[b]) % twok;
                        if (((bins >> (8 * b)) & 0xFFu) != wantbin) {
                            printf("FAIL bins k=%u act=%u v=%u got %u want %u\n", k, act, v[b], (bins >> (8 * b)) & 0xFFu,
                                   wantbin);
                            return 1;
                        }
                    }
                    checked++;
                }
            }
        }
        // Algorithm 3 in frame 0: the SWAR form against the scalar one, and the
        // scalar one against the paper's Algorithm 3 on the two maintained
        // blocks (ACT 0: i = -B, ACT k: i = k - B), through the per-block map.
        for (uint32_t B = 0; B < twok; B++) {
            const RangeConsts pc = preserve_consts_frame0(B, k);
            const uint32_t blk[2] = {(twok - B) % twok, (k + twok - B) % twok}, act[2] = {0u, k};
            for (uint32_t u = 0; u <= twok; u++)
                for (int z = 0; z < 2; z++) {
                    uint32_t got = to_canonical(preserve_frame0(u, B, k), blk[z], twok);
                    uint32_t want = preserve_at(to_canonical(u, blk[z], twok), act[z], k);
                    if (got != want || from_canonical(to_canonical(u, blk[z], twok), blk[z], twok) != u) {
                        printf("FAIL frame-0 preserve k=%u B=%u u=%u block=%u\n", k, B, u, blk[z]);
                        return 1;
                    }
                }
            for (int trial = 0; trial < 300; trial++) {
                uint32_t v[4];
                for (int b = 0; b < 4; b++) v[b] = rnd() % (twok + 1);
                uint32_t w = v[0] | v[1] << 8 | v[2] << 16 | v[3] << 24;
                uint32_t r = swar_preserve_frame0(w, pc, twok);
                for (int b = 0; b < 4; b++)
                    if (((r >> (8 * b)) & 0xFFu) != preserve_frame0(v[b], B, k)) {
                        printf("FAIL swar frame-0 preserve k=%u B=%u v=%u\n", k, B, v[b]);
                        return 1;
                    }
                checked++;
            }
        }
        // CheckAT and the distance of Eq. 5 read a frame-0 value with ACT = BACT^0
        // exactly as the paper's value with its block's ACT (Eq. 8)
        if (k == 1 || k == 2 || k == 5 || k == 10 || k == 33 || k == 63) {
            for (uint32_t B = 0; B < twok; B++)
                for (uint32_t i = 0; i < twok; i++)
                    for (uint32_t u = 0; u <= twok; u++)
                        for (uint32_t kp = 1; kp <= k; kp++) {
                            uint32_t v = to_canonical(u, i, twok), a = (B + i) % twok;
                            if (check_at(u, B, kp, twok) != check_at(v, a, kp, twok)) {
                                printf("FAIL frame-0 CheckAT k=%u B=%u i=%u u=%u k'=%u\n", k, B, i, u, kp);
                                return 1;
                            }
                        }
        }
    }
    // 16-bit ATs (k >= 64): CheckAT and CheckDR on two values per word
    const uint32_t wide[] = {64, 100, 300, 1023};
    for (uint32_t k : wide) {
        uint32_t twok = 2 * k, c2k = (0x8000u - twok) * ONES16;
        for (uint32_t act = 0; act < twok; act += (k > 100 ? 7 : 1)) {
            for (uint32_t kp = 1; kp <= k; kp += (k > 100 ? 13 : 1)) {
                RangeConsts rc = range_consts16(act, kp, twok), dc = dr_range_consts16(kp);
                for (int trial = 0; trial < 24; trial++) {
                    uint32_t v0 = rnd() % (twok + 1), v1 = rnd() % (twok + 1);
                    if (trial < 4) { v0 = trial & 1 ? twok : act; v1 = trial & 2 ? 0u : twok - 1u; }
                    uint32_t w = v0 | (v1 << 16);
                    uint32_t m = swar16_active(w, rc, c2k), d = swar16_active(w, dc, c2k);
                    bool g0 = (m >> 15) & 1u, g1 = (m >> 31) & 1u;
                    if (g0 != check_at(v0, act, kp, twok) || g1 != check_at(v1, act, kp, twok) ||
                        (((d >> 15) & 1u) != 0) != (v0 < kp && v0 <= k) || (((d >> 31) & 1u) != 0) != (v1 < kp && v1 <= k)) {
                        printf("FAIL swar16 k=%u act=%u k'=%u v=%u,%u\n", k, act, kp, v0, v1);
                        return 1;
                    }
                    checked++;
                }
            }
        }
    }
    printf("OK %ld words\n", checked);
    return 0;
}
