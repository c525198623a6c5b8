/*
 * ac_oracle.c -- plain serial CPU oracle for the Poisson-asynchronous Glauber
 * (continuous-time Ising) cellular array of Lubachevsky, "Efficient Parallel
 * Simulations of Asynchronous Cellular Arrays".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * definition that the GPU kernels are checked against.  Only the test suite,
 * the package smoke check and the benchmark's CPU-baseline leg may load it;
 * the library's product path never calls, links or includes it, and it
 * includes nothing from the library.
 *
 * What it computes (Sec. 1 "Poisson asynchrony"; Sec. 2, Eqs. (1)-(2)):
 *   every cell of a rows x cols torus owns an independent rate-1 Poisson
 *   clock; at each arrival the cell's spin is re-drawn by the Glauber
 *   heat-bath rule from the spins of its four neighbours just before the
 *   arrival.  The standard serial procedure of Sec. 1 (arrivals handled one
 *   at a time in global time order) with one random stream per cell
 *   (Sec. 3, invariance remark after Fig. 3.6) is implemented literally:
 *   a binary min-heap over the cells, keyed by (next-arrival tick, cell
 *   index), is popped until the top tick reaches t_end.
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes of the repository):
 *   R1 order   strict total order on (tick, row-major index); on equal
 *              ticks the smaller index goes first (the paper assumes no
 *              ties, Sec. 3 condition (ii)).
 *   R2 end     arrivals with tick < t_end are committed; after a run every
 *              cell's tick is its first uncommitted arrival, >= t_end
 *              (Fig. 3.1 loop condition "t(c) < end_time").
 *   R3 first   the first arrival is at t0 = exp_ticks(B(c,0).x) > 0, a
 *              plain Poisson process (the appendix program's extra event at
 *              time 0 is not reproduced).
 *   R4 random  Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
 *              (seed & 0xffffffff, seed >> 32).  Event block
 *              B(c,k) = Philox({c, k, 0, 0}); init block I(c) =
 *              Philox({c, 0, 1, 0}).  The commit of arrival n (n = 0,1,..)
 *              draws B(c, n+1): .y is its acceptance uniform and .x the gap
 *              to arrival n+1.  Random initial spin = +1 iff I(c).x is odd.
 *              This is the "each PE its own reproducible sequence" of
 *              Sec. 5, refined to one counter stream per cell.
 *   R5 gap     exp_ticks(x): an all-integer stand-in for -ln r in Eq. (5)
 *              with 2^32 ticks per unit time (see exp_ticks below).
 *   R6 table   p = 1 / (1 + exp(beta * dE)), dE = 2 s (J S + h), in IEEE
 *              binary64; thr = min(floor(p * 2^32), 2^32 - 1); flip iff
 *              u32 < thr.  Same probabilities as the appendix's x/(1+x),
 *              x = exp(-dE/T).  Index j + 5*(s > 0), j = number of up
 *              neighbours, as in the appendix's prob[10].
 *   R7 nbrs    4 nearest neighbours on the periodic torus, counted with
 *              multiplicity (on a 2-wide torus both sides are one cell).
 *   R11 laws   time-only model of Sec. 4: exponential (R5), uniform on
 *              (0, 1] as x + 1 ticks, and r^(1/8) as three nested integer
 *              square roots (see aco_gap below).
 *   R12 life   Life-like rules: Moore neighbourhood, birth / survival masks
 *              over the live-neighbour count (see aco_life_run below).
 *   R13 rates  per-cell rates of law (A): gap scaled by m_c / 2^20 (see
 *              aco_rated_gap below).
 *   R14 q-nbhd the Ising array on the q-th degree neighbourhood (see
 *              aco_run_q below).
 *
 * Build: plain C99 + libm, -O2 -ffp-contract=off (no fused multiply-add, so
 * the binary64 table is the same on every host).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. on the Philox family).   */
/* One round: two 32x32->64 products of the even counter words with   */
/* the round multipliers; the high halves are xored with the odd words */
/* and the round key, the words are permuted; the key is bumped by the */
/* Weyl increments between rounds.                                     */
/* ------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void aco_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_block(uint64_t seed, uint32_t c, uint32_t w1, uint32_t w2, uint32_t out[4])
{
    uint32_t ctr[4] = {c, w1, w2, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    aco_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------ */
/* exp_ticks(x): integer exponential gap, reading R5.                  */
/*   m  = 2x + 1 (odd), so u = m / 2^33 lies strictly inside (0, 1);   */
/*   k  = floor(log2 m);  y = m scaled to a Q1.31 mantissa in           */
/*        [2^31, 2^32) (truncating when k = 32);                        */
/*   32 fraction bits of log2(y / 2^31) by repeated squaring: square,   */
/*        keep Q1.31 (truncate), and when the square reaches 2 emit a   */
/*        1 bit and halve (the textbook bit-by-bit binary logarithm);   */
/*   lg = k + f / 2^32 ~ log2 m;  nl = 33 - lg ~ -log2 u  (Q.32, >= 1); */
/*   gap = floor(nl * ln2 * 2^64 / 2^64) + 1 ticks, with               */
/*        LN2_Q64 = floor(ln 2 * 2^64) and an exact 128-bit product.   */
/* The +1 keeps next_t > t (Eq. (2)).                                  */
/* ------------------------------------------------------------------ */
#define LN2_Q64 0xB17217F7D1CF79ABull

uint64_t aco_exp_ticks(uint32_t x)
{
    uint64_t m = 2ull * (uint64_t)x + 1ull;
    int k = 0;
    while ((m >> (k + 1)) != 0) ++k;            /* k = floor(log2 m), 0..32 */
    uint64_t y = (k >= 31) ? (m >> (k - 31)) : (m << (31 - k));
    uint64_t f = 0;
    for (int i = 0; i < 32; ++i) {
        y = (y * y) >> 31;
        f <<= 1;
        if (y >= (1ull << 32)) {
            y >>= 1;
            f |= 1ull;
        }
    }
    uint64_t lg = ((uint64_t)k << 32) | f;
    uint64_t nl = (33ull << 32) - lg;
    unsigned __int128 prod = (unsigned __int128)nl * (unsigned __int128)LN2_Q64;
    return (uint64_t)(prod >> 64) + 1ull;
}

/* ------------------------------------------------------------------ */
/* Flip-threshold table, reading R6 (appendix, flip probabilities).   */
/* ------------------------------------------------------------------ */
void aco_thresholds(double beta, double J, double h, uint32_t thr[10])
{
    for (int sp = 0; sp < 2; ++sp) {
        double s = sp ? 1.0 : -1.0;
        for (int j = 0; j < 5; ++j) {
            double S = (double)(2 * j - 4);
            double dE = 2.0 * s * (J * S + h);
            double p = 1.0 / (1.0 + exp(beta * dE));
            double v = ldexp(p, 32);
            uint32_t t;
            if (!(v < 4294967295.0))
                t = 0xFFFFFFFFu;          /* p = 1 (or NaN): saturate */
            else
                t = (uint32_t)floor(v);
            thr[j + 5 * sp] = t;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Initial state (readings R3, R4).  init: 0 random, 1 all up, 2 down. */
/* ------------------------------------------------------------------ */
void aco_init(int32_t rows, int32_t cols, int32_t init, uint64_t seed,
              int8_t *s, int64_t *t, uint32_t *n)
{
    uint64_t N = (uint64_t)rows * (uint64_t)cols;
    for (uint64_t c = 0; c < N; ++c) {
        uint32_t b0[4], ib[4];
        philox_block(seed, (uint32_t)c, 0u, 0u, b0);
        if (init == 1)
            s[c] = 1;
        else if (init == 2)
            s[c] = -1;
        else {
            philox_block(seed, (uint32_t)c, 0u, 1u, ib);
            s[c] = (ib[0] & 1u) ? 1 : -1;
        }
        t[c] = (int64_t)aco_exp_ticks(b0[0]);
        n[c] = 0u;
    }
}

/* Torus neighbours of c in the order up, down, left, right. */
static void neighbours(int32_t rows, int32_t cols, uint64_t c, uint64_t nb[4])
{
    int64_t r = (int64_t)(c / (uint64_t)cols), q = (int64_t)(c % (uint64_t)cols);
    nb[0] = (uint64_t)(((r - 1 + rows) % rows) * cols + q);
    nb[1] = (uint64_t)(((r + 1) % rows) * cols + q);
    nb[2] = (uint64_t)(r * cols + (q - 1 + cols) % cols);
    nb[3] = (uint64_t)(r * cols + (q + 1) % cols);
}

/* ------------------------------------------------------------------ */
/* Binary min-heap over cells keyed by (t[c], c)  (reading R1).        */
/* ------------------------------------------------------------------ */
static int key_less(const int64_t *t, uint32_t a, uint32_t b)
{
    return (t[a] < t[b]) || (t[a] == t[b] && a < b);
}

static void sift_down(uint32_t *heap, uint64_t size, uint64_t i, const int64_t *t)
{
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < size && key_less(t, heap[l], heap[m])) m = l;
        if (r < size && key_less(t, heap[r], heap[m])) m = r;
        if (m == i) return;
        uint32_t tmp = heap[i]; heap[i] = heap[m]; heap[m] = tmp;
        i = m;
    }
}

/*
 * Continue the trajectory from state (s, t, n) until every cell's next
 * arrival is >= t_end (reading R2).  Returns the number of committed
 * arrivals, or -1 if the heap could not be allocated.
 */
uint64_t aco_rated_gap(uint64_t e, uint32_t m);

/* The heap run; m = NULL for rate 1 everywhere, else per-cell rates (R13). */
static int64_t run_heap(int32_t rows, int32_t cols, const uint32_t thr[10], uint64_t seed, const uint32_t *m,
                        int8_t *s, int64_t *t, uint32_t *n, int64_t t_end)
{
    uint64_t N = (uint64_t)rows * (uint64_t)cols;
    uint32_t *heap = (uint32_t *)malloc(N * sizeof(uint32_t));
    if (!heap) return -1;
    for (uint64_t c = 0; c < N; ++c) heap[c] = (uint32_t)c;
    for (uint64_t i = N / 2; i-- > 0;) sift_down(heap, N, i, t);

    int64_t events = 0;
    while (t[heap[0]] < t_end) {
        uint32_t c = heap[0];
        uint64_t nb[4];
        neighbours(rows, cols, c, nb);
        int up = 0;                                   /* spins just before t(c) */
        for (int d = 0; d < 4; ++d) up += (s[nb[d]] > 0);
        uint32_t b[4];
        philox_block(seed, c, n[c] + 1u, 0u, b);
        if (b[1] < thr[up + 5 * (s[c] > 0)]) s[c] = (int8_t)(-s[c]);  /* Eq. (1) */
        uint64_t gap = aco_exp_ticks(b[0]);                            /* Eq. (5) */
        t[c] += (int64_t)(m ? aco_rated_gap(gap, m[c]) : gap);
        n[c] += 1u;
        sift_down(heap, N, 0, t);
        ++events;
    }
    free(heap);
    return events;
}

int64_t aco_run(int32_t rows, int32_t cols, const uint32_t thr[10], uint64_t seed,
                int8_t *s, int64_t *t, uint32_t *n, int64_t t_end)
{
    return run_heap(rows, cols, thr, seed, NULL, s, t, n, t_end);
}

/* ------------------------------------------------------------------ */
/* Per-cell rates: the general asynchrony law (A) of Sec. 2, next       */
/* arrival t - ln(r) / p_c.  Reading R13: p_c = 2^20 / m_c for a 32-bit  */
/* multiplier m_c >= 1, and the gap is                                  */
/*   max(1, floor(exp_ticks(x) * m_c / 2^20))                           */
/* (m_c = 2^20 is the rate-1 process of R5 exactly).  The first arrival */
/* uses the same scaling of B(c,0).x.                                   */
/* ------------------------------------------------------------------ */
uint64_t aco_rated_gap(uint64_t e, uint32_t m)
{
    unsigned __int128 p = (unsigned __int128)e * (unsigned __int128)m;
    uint64_t g = (uint64_t)(p >> 20);
    return g ? g : 1u;
}

void aco_init_rated(int32_t rows, int32_t cols, int32_t init, uint64_t seed, const uint32_t *m,
                    int8_t *s, int64_t *t, uint32_t *n)
{
    aco_init(rows, cols, init, seed, s, t, n);
    uint64_t N = (uint64_t)rows * (uint64_t)cols;
    for (uint64_t c = 0; c < N; ++c) t[c] = (int64_t)aco_rated_gap((uint64_t)t[c], m[c]);
}

int64_t aco_run_rated(int32_t rows, int32_t cols, const uint32_t thr[10], uint64_t seed, const uint32_t *m,
                      int8_t *s, int64_t *t, uint32_t *n, int64_t t_end)
{
    return run_heap(rows, cols, thr, seed, m, s, t, n, t_end);
}

/* ------------------------------------------------------------------ */
/* The Ising array on the q-th degree neighbourhood of Sec. 3 (reading  */
/* R14): every cell within Manhattan distance q is a neighbour, M =     */
/* 2q(q+1) of them; the heat-bath rule of R6 with S = sum of their      */
/* spins (S = 2j - M for j up neighbours), table index j + (M+1)(s>0),  */
/* and a cell waits for all of them.  q = 1 is the model above.  Needs  */
/* rows, cols >= 2q + 1 (distinct neighbours).                          */
/* ------------------------------------------------------------------ */
void aco_thresholds_q(double beta, double J, double h, int32_t q, uint32_t *thr)
{
    const int M = 2 * q * (q + 1);
    for (int sp = 0; sp < 2; ++sp) {
        double s = sp ? 1.0 : -1.0;
        for (int j = 0; j <= M; ++j) {
            double S = (double)(2 * j - M);
            double p = 1.0 / (1.0 + exp(beta * 2.0 * s * (J * S + h)));
            double v = ldexp(p, 32);
            thr[j + (M + 1) * sp] = (v < 4294967295.0) ? (uint32_t)floor(v) : 0xFFFFFFFFu;
        }
    }
}

int64_t aco_run_q(int32_t rows, int32_t cols, int32_t q, const uint32_t *thr, uint64_t seed,
                  int8_t *s, int64_t *t, uint32_t *n, int64_t t_end)
{
    const int M = 2 * q * (q + 1);
    uint64_t N = (uint64_t)rows * (uint64_t)cols;
    uint32_t *heap = (uint32_t *)malloc(N * sizeof(uint32_t));
    if (!heap) return -1;
    for (uint64_t c = 0; c < N; ++c) heap[c] = (uint32_t)c;
    for (uint64_t i = N / 2; i-- > 0;) sift_down(heap, N, i, t);
    int64_t events = 0;
    while (t[heap[0]] < t_end) {
        uint32_t c = heap[0];
        int64_t r = (int64_t)(c / (uint32_t)cols), x = (int64_t)(c % (uint32_t)cols);
        int up = 0;
        for (int dr = -q; dr <= q; ++dr)
            for (int dx = -q; dx <= q; ++dx) {
                int dist = (dr < 0 ? -dr : dr) + (dx < 0 ? -dx : dx);
                if (dist == 0 || dist > q) continue;
                up += s[((r + dr + rows) % rows) * cols + (x + dx + cols) % cols] > 0;
            }
        uint32_t b[4];
        philox_block(seed, c, n[c] + 1u, 0u, b);
        if (b[1] < thr[up + (M + 1) * (s[c] > 0)]) s[c] = (int8_t)(-s[c]);
        t[c] += (int64_t)aco_exp_ticks(b[0]);
        n[c] += 1u;
        sift_down(heap, N, 0, t);
        ++events;
    }
    free(heap);
    return events;
}

/* ------------------------------------------------------------------ */
/* Asynchronous Life-like automaton (Sec. 3: the deterministic update   */
/* under Poisson asynchrony, with Conway's Game of Life as the example  */
/* of a rule that leaves most cells unchanged).  Reading R12: the       */
/* neighbourhood is the 8-cell Moore neighbourhood on the torus; at an  */
/* arrival a cell with k live neighbours becomes                        */
/*   alive ? bit k of `survive` : bit k of `birth`                      */
/* (Conway: birth = 1<<3, survive = 1<<2 | 1<<3), from the states just  */
/* before the arrival; arrivals are the same Poisson process as for the */
/* Ising array (R3-R5: first gap from B(c,0).x, the commit of arrival n */
/* advances by exp_ticks(B(c,n+1).x)).  Initial state: alive iff        */
/* I(c).x < density (init 0), all alive (1), all dead (2).  Alive is    */
/* s = +1, dead s = -1.  Needs rows, cols >= 3 (8 distinct neighbours). */
/* ------------------------------------------------------------------ */
void aco_life_init(int32_t rows, int32_t cols, int32_t init, uint32_t density, uint64_t seed,
                   int8_t *s, int64_t *t, uint32_t *n)
{
    uint64_t N = (uint64_t)rows * (uint64_t)cols;
    for (uint64_t c = 0; c < N; ++c) {
        uint32_t b0[4], ib[4];
        philox_block(seed, (uint32_t)c, 0u, 0u, b0);
        if (init == 1)
            s[c] = 1;
        else if (init == 2)
            s[c] = -1;
        else {
            philox_block(seed, (uint32_t)c, 0u, 1u, ib);
            s[c] = (ib[0] < density) ? 1 : -1;
        }
        t[c] = (int64_t)aco_exp_ticks(b0[0]);
        n[c] = 0u;
    }
}

int64_t aco_life_run(int32_t rows, int32_t cols, uint32_t birth, uint32_t survive, uint64_t seed,
                     int8_t *s, int64_t *t, uint32_t *n, int64_t t_end)
{
    uint64_t N = (uint64_t)rows * (uint64_t)cols;
    uint32_t *heap = (uint32_t *)malloc(N * sizeof(uint32_t));
    if (!heap) return -1;
    for (uint64_t c = 0; c < N; ++c) heap[c] = (uint32_t)c;
    for (uint64_t i = N / 2; i-- > 0;) sift_down(heap, N, i, t);

    int64_t events = 0;
    while (t[heap[0]] < t_end) {
        uint32_t c = heap[0];
        int64_t r = (int64_t)(c / (uint32_t)cols), q = (int64_t)(c % (uint32_t)cols);
        int k = 0;                                    /* live Moore neighbours */
        for (int dr = -1; dr <= 1; ++dr)
            for (int dq = -1; dq <= 1; ++dq) {
                if (dr == 0 && dq == 0) continue;
                int64_t rr = (r + dr + rows) % rows, qq = (q + dq + cols) % cols;
                k += (s[rr * cols + qq] > 0);
            }
        uint32_t mask = (s[c] > 0) ? survive : birth;
        s[c] = ((mask >> k) & 1u) ? 1 : -1;
        uint32_t b[4];
        philox_block(seed, c, n[c] + 1u, 0u, b);
        t[c] += (int64_t)aco_exp_ticks(b[0]);
        n[c] += 1u;
        sift_down(heap, N, 0, t);
        ++events;
    }
    free(heap);
    return events;
}

/* ------------------------------------------------------------------ */
/* Time-only round model of Sec. 4 applied to the synchronous          */
/* one-cell-per-PE algorithm (Fig. 3.2): in each round every cell whose */
/* key is below all of its neighbours' keys and whose tick is < t_end   */
/* advances its time; only times are tracked (for the Ising law the     */
/* next arrival does not depend on the spins).  The per-round number of */
/* advancing cells is written to enabled[] (up to max_rounds entries).  */
/* Returns the number of rounds with at least one advancing cell.       */
/* ------------------------------------------------------------------ */
int64_t aco_time_rounds(int32_t rows, int32_t cols, uint64_t seed, int64_t *t, uint32_t *n,
                        int64_t t_end, int64_t max_rounds, int64_t *enabled)
{
    uint64_t N = (uint64_t)rows * (uint64_t)cols;
    uint8_t *en = (uint8_t *)malloc(N);
    if (!en) return -1;
    int64_t rounds = 0;
    for (;;) {
        int64_t cnt = 0;
        for (uint64_t c = 0; c < N; ++c) {
            uint64_t nb[4];
            neighbours(rows, cols, c, nb);
            int ok = t[c] < t_end;
            for (int d = 0; d < 4 && ok; ++d)
                if (!key_less(t, (uint32_t)c, (uint32_t)nb[d])) ok = 0;
            en[c] = (uint8_t)ok;
            cnt += ok;
        }
        if (cnt == 0) break;
        for (uint64_t c = 0; c < N; ++c) {
            if (!en[c]) continue;
            uint32_t b[4];
            philox_block(seed, (uint32_t)c, n[c] + 1u, 0u, b);
            t[c] += (int64_t)aco_exp_ticks(b[0]);
            n[c] += 1u;
        }
        if (rounds < max_rounds) enabled[rounds] = cnt;
        ++rounds;
    }
    free(en);
    return rounds;
}

/* ------------------------------------------------------------------ */
/* Time-only round model in one, two and three dimensions (Sec. 4: the  */
/* six experiments behind the one-cell-per-PE efficiency figure -- an   */
/* n-cell circle, an n x n torus and an n x n x n periodic array, with  */
/* exponential or uniform increments, and the r^(1/8) increments of the */
/* same section).  Times only: a cell advances in a round iff its key   */
/* (t, index) is below the keys of all its neighbours -- the 2*dims     */
/* nearest ones, or every cell within Manhattan distance q for the q-th */
/* degree neighbourhood of Sec. 3 (n >= 2q+1) -- (R1) and t < t_end;    */
/* advancing cells draw their next increment afterwards.                */
/*                                                                      */
/* Increment laws (reading R11), from the 32-bit word x = B(c, k).x:    */
/*   0  exponential: exp_ticks(x) (R5)                                  */
/*   1  uniform on (0, 1]: x + 1 ticks                                  */
/*   2  r^(1/8), r = (2x+1)/2^33 uniform on (0, 1): three nested        */
/*      integer square roots, s1 = isqrt((2x+1) 2^31) = floor(2^32 r^   */
/*      (1/2)), s2 = isqrt(s1 2^32), gap = isqrt(s2 2^32)               */
/* Initial times t0 = gap(B(c, 0).x) as in R3; cell c's k-th advance     */
/* draws B(c, k).x.  Cell index: row-major, ((z n) + y) n + x.          */
/* ------------------------------------------------------------------ */

/* floor(sqrt(v)), the digit-by-digit (base 4) method */
static uint64_t isqrt64(uint64_t v)
{
    uint64_t res = 0, bit = 1ull << 62;
    while (bit > v) bit >>= 2;
    while (bit) {
        if (v >= res + bit) {
            v -= res + bit;
            res = (res >> 1) + bit;
        } else {
            res >>= 1;
        }
        bit >>= 2;
    }
    return res;
}

uint64_t aco_gap(int32_t law, uint32_t x)
{
    if (law == 0) return aco_exp_ticks(x);
    if (law == 1) return (uint64_t)x + 1ull;
    uint64_t s1 = isqrt64((2ull * (uint64_t)x + 1ull) << 31);
    uint64_t s2 = isqrt64(s1 << 32);
    return isqrt64(s2 << 32);
}

/* The q-th degree neighbourhood of Sec. 3 (neighbours of neighbours, q times):   */
/* every cell within Manhattan distance 1..q on the periodic array.  Writes the   */
/* neighbour indices to nb[] and returns their number (2 dims for q = 1).         */
static int neighbours_nd(int32_t dims, int64_t n, int32_t q, uint64_t c, uint64_t *nb)
{
    int64_t coord[3] = {0, 0, 0}, stride[3] = {1, n, n * n};
    uint64_t rest = c;
    for (int a = 0; a < dims; ++a) {
        coord[a] = (int64_t)(rest % (uint64_t)n);
        rest /= (uint64_t)n;
    }
    int m = 0;
    int64_t lim[3] = {q, dims > 1 ? q : 0, dims > 2 ? q : 0};
    for (int64_t dz = -lim[2]; dz <= lim[2]; ++dz)
        for (int64_t dy = -lim[1]; dy <= lim[1]; ++dy)
            for (int64_t dx = -lim[0]; dx <= lim[0]; ++dx) {
                int64_t dist = (dx < 0 ? -dx : dx) + (dy < 0 ? -dy : dy) + (dz < 0 ? -dz : dz);
                if (dist == 0 || dist > q) continue;
                int64_t d[3] = {dx, dy, dz};
                uint64_t idx = 0;
                for (int a = 0; a < dims; ++a)
                    idx += (uint64_t)(((coord[a] + d[a]) % n + n) % n * stride[a]);
                nb[m++] = idx;
            }
    return m;
}

int64_t aco_time_model(int32_t dims, int64_t n, int32_t q, int32_t law, uint64_t seed, int64_t t_end,
                       int64_t max_rounds, int64_t *enabled, int64_t *t_out, uint32_t *n_out)
{
    if (dims < 1 || dims > 3 || n < 2 || law < 0 || law > 2 || q < 1 || q > 8 || (q > 1 && n < 2 * q + 1))
        return -2;
    uint64_t N = (uint64_t)n;
    for (int a = 1; a < dims; ++a) N *= (uint64_t)n;
    int64_t *t = (int64_t *)malloc(N * sizeof(int64_t));
    uint32_t *cnt = (uint32_t *)calloc(N, sizeof(uint32_t));
    uint8_t *en = (uint8_t *)malloc(N);
    if (!t || !cnt || !en) {
        free(t); free(cnt); free(en);
        return -1;
    }
    for (uint64_t c = 0; c < N; ++c) {
        uint32_t b[4];
        philox_block(seed, (uint32_t)c, 0u, 0u, b);
        t[c] = (int64_t)aco_gap(law, b[0]);
    }
    int64_t rounds = 0;
    while (rounds < max_rounds) {
        int64_t nen = 0;
        for (uint64_t c = 0; c < N; ++c) {
            uint64_t nb[2 * 8 * 9 * 17];
            int m = neighbours_nd(dims, n, q, c, nb);
            int ok = t[c] < t_end;
            for (int d = 0; d < m && ok; ++d)
                if (nb[d] != c && !key_less(t, (uint32_t)c, (uint32_t)nb[d])) ok = 0;
            en[c] = (uint8_t)ok;
            nen += ok;
        }
        if (nen == 0) break;
        for (uint64_t c = 0; c < N; ++c) {
            if (!en[c]) continue;
            uint32_t b[4];
            philox_block(seed, (uint32_t)c, cnt[c] + 1u, 0u, b);
            t[c] += (int64_t)aco_gap(law, b[0]);
            cnt[c] += 1u;
        }
        enabled[rounds] = nen;
        ++rounds;
    }
    if (t_out) memcpy(t_out, t, N * sizeof(int64_t));
    if (n_out) memcpy(n_out, cnt, N * sizeof(uint32_t));
    free(t); free(cnt); free(en);
    return rounds;
}

/* ------------------------------------------------------------------ */
/* Observables and a state fingerprint.                                */
/* Energy  E = -J sum_bonds s s' - h sum s  over right and down bonds   */
/* (appendix, energy comment), with the same multiplicity as the        */
/* neighbour sum.  out[0] = sum s, out[1] = sum over bonds of s s'.     */
/* ------------------------------------------------------------------ */
void aco_observables(int32_t rows, int32_t cols, const int8_t *s, int64_t out[2])
{
    int64_t m = 0, b = 0;
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t q = 0; q < cols; ++q) {
            int64_t c = r * cols + q;
            m += s[c];
            b += (int64_t)s[c] * s[r * cols + (q + 1) % cols];
            b += (int64_t)s[c] * s[((r + 1) % rows) * cols + q];
        }
    out[0] = m;
    out[1] = b;
}

/* BKL classes (Sec. 3, "The BKL algorithm"): the heat-bath flip probability of */
/* a cell depends only on its spin and its number j of up neighbours, so the     */
/* cells fall into 10 classes, index j + 5 (s > 0) as in the threshold table.   */
/* out[k] = number of cells in class k.                                         */
void aco_class_counts(int32_t rows, int32_t cols, const int8_t *s, int64_t out[10])
{
    for (int k = 0; k < 10; ++k) out[k] = 0;
    uint64_t N = (uint64_t)rows * (uint64_t)cols;
    for (uint64_t c = 0; c < N; ++c) {
        uint64_t nb[4];
        neighbours(rows, cols, c, nb);
        int up = 0;
        for (int d = 0; d < 4; ++d) up += (s[nb[d]] > 0);
        out[up + 5 * (s[c] > 0)] += 1;
    }
}

/* SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA'14) used as a mixer. */
static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/*
 * Order-independent fingerprint of a full state:
 *   sum over cells c of mix(mix(mix(c) ^ t[c]) ^ (2 n[c] + [s[c] > 0]))  (mod 2^64).
 */
uint64_t aco_checksum(int32_t rows, int32_t cols, const int8_t *s, const int64_t *t,
                      const uint32_t *n)
{
    uint64_t N = (uint64_t)rows * (uint64_t)cols, acc = 0;
    for (uint64_t c = 0; c < N; ++c) {
        uint64_t z = mix64(c);
        z = mix64(z ^ (uint64_t)t[c]);
        z = mix64(z ^ ((uint64_t)n[c] << 1 | (uint64_t)(s[c] > 0)));
        acc += z;
    }
    return acc;
}

/* ------------------------------------------------------------------ */
/* Batch helpers for tests (loops over the scalar definitions above).  */
/* ------------------------------------------------------------------ */
void aco_exp_ticks_many(const uint32_t *x, uint64_t *out, int64_t count)
{
    for (int64_t i = 0; i < count; ++i) out[i] = aco_exp_ticks(x[i]);
}

/* out[4*i .. 4*i+3] = Philox({c[i], k[i], w2, 0}) under the seed's key. */
void aco_philox_blocks(uint64_t seed, const uint32_t *c, const uint32_t *k, uint32_t w2,
                       uint32_t *out, int64_t count)
{
    for (int64_t i = 0; i < count; ++i) philox_block(seed, c[i], k[i], w2, out + 4 * i);
}
