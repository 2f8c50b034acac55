/*
 * CPU ORACLE companions (test infrastructure only):
 *   - the paper's accelerated scheme "ALDP" (Sec. 2.3): Kirsch responses from
 *     fifteen shared column partial sums A0..A14 (Eqs. 7-21) combined three
 *     at a time (Eqs. 22-29).  It is a second, independent formula for m_i,
 *     used to pin the mask orientation of oracle_ldp.c, and the timed CPU
 *     port of the paper's method.
 *   - the ring-sum identity m_i = 8*S3_i - 3*S8 written out on the CPU.
 *   - an independent formulation of Eq. 2 by rank counting.
 *
 * Four of the printed column sums are garbled; the readings used below are
 * the ones that make Eqs. 22-29 reproduce Kirsch compass masks:
 *   A7  (Eq. 14) = 5(I(x-1,y-1) + I(x,y-1)) - 3 I(x+1,y-1)    left column of M3
 *   A9  (Eq. 16) = 5(I(x-1,y-1) + I(x,y-1) + I(x+1,y-1))      left column of M4
 *   A11 (Eq. 18) = -3 I(x-1,y) + 5 I(x+1,y)                   middle column of M5..M7
 *   A12 (Eq. 19) = -3(I(x-1,y-1) + I(x,y-1)) + 5 I(x+1,y-1)   left column of M6
 * x is the row and y the column, as in Eq. 1.
 */
#include "oracle_ldp.h"

#include <stddef.h>

#define P(dx, dy) ((int32_t)img[(size_t)(x + (dx)) * (size_t)pitch + (size_t)(y + (dy))])

void aldp_responses(const uint8_t *img, int H, int W, int pitch, int x, int y, int32_t m[8]) {
    (void)H;
    (void)W;
    /* Kirsch mask reconstruction, Sec. 2.3.1 (Eqs. 7-21). */
    const int32_t A0 = -3 * (P(-1, -1) + P(0, -1) + P(1, -1));          /* Eq. 7  */
    const int32_t A1 = -3 * (P(-1, 0) + P(1, 0));                      /* Eq. 8  */
    const int32_t A2 = 5 * (P(-1, 1) + P(0, 1) + P(1, 1));             /* Eq. 9  */
    const int32_t A3 = 5 * P(-1, 0) - 3 * P(1, 0);                     /* Eq. 10 */
    const int32_t A4 = 5 * (P(-1, 1) + P(0, 1)) - 3 * P(1, 1);         /* Eq. 11 */
    const int32_t A5 = 5 * P(-1, -1) - 3 * (P(0, -1) + P(1, -1));      /* Eq. 12 */
    const int32_t A6 = 5 * P(-1, 1) - 3 * (P(0, 1) + P(1, 1));         /* Eq. 13 */
    const int32_t A7 = 5 * (P(-1, -1) + P(0, -1)) - 3 * P(1, -1);      /* Eq. 14, corrected */
    const int32_t A8 = -3 * (P(-1, 1) + P(0, 1) + P(1, 1));            /* Eq. 15 */
    const int32_t A9 = 5 * (P(-1, -1) + P(0, -1) + P(1, -1));          /* Eq. 16, corrected */
    const int32_t A10 = -3 * P(-1, -1) + 5 * (P(0, -1) + P(1, -1));    /* Eq. 17 */
    const int32_t A11 = -3 * P(-1, 0) + 5 * P(1, 0);                   /* Eq. 18, corrected */
    const int32_t A12 = -3 * (P(-1, -1) + P(0, -1)) + 5 * P(1, -1);    /* Eq. 19, corrected */
    const int32_t A13 = -3 * (P(-1, 1) + P(0, 1)) + 5 * P(1, 1);       /* Eq. 20 */
    const int32_t A14 = -3 * P(-1, 1) + 5 * (P(0, 1) + P(1, 1));       /* Eq. 21 */
    /* Edge response calculation, Sec. 2.3.2 (Eqs. 22-29). */
    m[0] = A0 + A1 + A2;    /* Eq. 22 */
    m[1] = A0 + A3 + A4;    /* Eq. 23 */
    m[2] = A5 + A3 + A6;    /* Eq. 24 */
    m[3] = A7 + A3 + A8;    /* Eq. 25 */
    m[4] = A9 + A1 + A8;    /* Eq. 26 */
    m[5] = A10 + A11 + A8;  /* Eq. 27 */
    m[6] = A12 + A11 + A13; /* Eq. 28 */
    m[7] = A0 + A11 + A14;  /* Eq. 29 */
}

/* Each Kirsch mask weighs ring positions i-1, i, i+1 by 5 and the other five
 * by -3, so m_i = 5*S3_i - 3*(S8 - S3_i) = 8*S3_i - 3*S8, where the ring
 * p_0..p_7 runs counter-clockwise from East. */
void ringsum_responses(const uint8_t *img, int H, int W, int pitch, int x, int y, int32_t m[8]) {
    (void)H;
    (void)W;
    const int32_t p[8] = {P(0, 1), P(-1, 1), P(-1, 0), P(-1, -1), P(0, -1), P(1, -1), P(1, 0), P(1, 1)};
    int32_t s8 = 0;
    for (int j = 0; j < 8; ++j) s8 += p[j];
    for (int i = 0; i < 8; ++i) m[i] = 8 * (p[(i + 7) & 7] + p[i] + p[(i + 1) & 7]) - 3 * s8;
}

#undef P

static inline int32_t iabs32(int32_t v) { return v < 0 ? -v : v; }

int rank_code_from_responses(const int32_t m[8], int k) {
    int code = 0;
    for (int i = 0; i < 8; ++i) {
        int beaten_by = 0;
        for (int j = 0; j < 8; ++j) {
            if (j == i) continue;
            int32_t a = iabs32(m[j]), b = iabs32(m[i]);
            if (a > b || (a == b && j < i)) ++beaten_by;
        }
        if (beaten_by < k) code |= 1 << i;
    }
    return code;
}

int aldp_codes(const uint8_t *img, int H, int W, int pitch, int k, uint8_t *codes, int code_pitch) {
    if (!img || !codes || H < 3 || W < 3 || pitch < W || k < 1 || k > 7) return -1;
    for (int x = 1; x < H - 1; ++x)
        for (int y = 1; y < W - 1; ++y) {
            int32_t m[8];
            aldp_responses(img, H, W, pitch, x, y, m);
            codes[(size_t)(x - 1) * code_pitch + (size_t)(y - 1)] = (uint8_t)rank_code_from_responses(m, k);
        }
    return 0;
}
