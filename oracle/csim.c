/*
 * Oracle hot loops in plain C (test infrastructure, loaded with ctypes by oracle/csim.py).
 * Not part of the product: shares no code with paper_2412_14975_gb300/ and is never linked
 * into it.
 *
 * 1. oracle_thompson_accept -- Thompson state-set simulation (the serial device operation of
 *    Sec. 2 with a nondeterministic recognizer): S <- eps-closure({start}); per byte
 *    S <- eps-closure(move(S, b)); accept <=> MATCH in S.  The closure is a plain depth-first
 *    walk over split states with a generation mark per state (no precomputed tables).
 *
 * 2. oracle_set_run -- rho extended to strings over an epsilon-free NFA (the position NFA):
 *    S <- (U_{q in S} follow[q]) n sym[b], from a given start set (proof of Th. 1, where
 *    rho(q, x) is the set of states reached from q after x).  Used for the chunk mappings
 *    lambda_i(a) = rho(q_a, y_i) (Lemma 1) at sizes too large for Python.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { K_CHAR = 0, K_SPLIT = 1, K_MATCH = 2 };

/* kind[n], out1[n], out2[n], sym[n*32] (256-bit byte set per state, bit b of byte b/8). */
int oracle_thompson_accept(int32_t n, const uint8_t *kind, const int32_t *out1,
                           const int32_t *out2, const uint8_t *sym, int32_t start,
                           const uint8_t *text, int64_t len)
{
    int32_t *cur = malloc(sizeof(int32_t) * n), *nxt = malloc(sizeof(int32_t) * n);
    int32_t *stack = malloc(sizeof(int32_t) * n);
    uint32_t *mark = calloc((size_t)n, sizeof(uint32_t));
    if (!cur || !nxt || !stack || !mark) {
        free(cur); free(nxt); free(stack); free(mark);
        return -1;
    }
    uint32_t gen = 1;
    int32_t ncur = 0, nnxt;

    /* add s and its eps-closure to list (one generation per step) */
#define ADD_CLOSURE(list, cnt, s0)                                         \
    do {                                                                   \
        int32_t sp = 0;                                                    \
        if ((s0) >= 0 && mark[(s0)] != gen) { mark[(s0)] = gen; stack[sp++] = (s0); } \
        while (sp > 0) {                                                   \
            int32_t s = stack[--sp];                                       \
            if (kind[s] == K_SPLIT) {                                      \
                int32_t t1 = out1[s], t2 = out2[s];                        \
                if (t1 >= 0 && mark[t1] != gen) { mark[t1] = gen; stack[sp++] = t1; } \
                if (t2 >= 0 && mark[t2] != gen) { mark[t2] = gen; stack[sp++] = t2; } \
            } else {                                                       \
                list[(cnt)++] = s;                                         \
            }                                                              \
        }                                                                  \
    } while (0)

    ADD_CLOSURE(cur, ncur, start);
    for (int64_t i = 0; i < len && ncur > 0; ++i) {
        const uint8_t b = text[i];
        ++gen;
        nnxt = 0;
        for (int32_t j = 0; j < ncur; ++j) {
            int32_t s = cur[j];
            if (kind[s] == K_CHAR && (sym[(size_t)s * 32 + (b >> 3)] >> (b & 7)) & 1)
                ADD_CLOSURE(nxt, nnxt, out1[s]);
        }
        int32_t *t = cur; cur = nxt; nxt = t;
        ncur = nnxt;
    }
    int acc = 0;
    for (int32_t j = 0; j < ncur; ++j)
        if (kind[cur[j]] == K_MATCH) acc = 1;
#undef ADD_CLOSURE
    free(cur); free(nxt); free(stack); free(mark);
    return acc;
}

/* follow[n*words], sym[256*words], start[words] -> out[words]; returns 1 if out is non-empty. */
int oracle_set_run(int32_t n, int32_t words, const uint64_t *follow, const uint64_t *sym,
                   const uint64_t *start, const uint8_t *text, int64_t len, uint64_t *out)
{
    uint64_t *cur = malloc(sizeof(uint64_t) * words), *nxt = malloc(sizeof(uint64_t) * words);
    if (!cur || !nxt) { free(cur); free(nxt); return -1; }
    memcpy(cur, start, sizeof(uint64_t) * words);
    int live = 0;
    for (int32_t w = 0; w < words; ++w) live |= cur[w] != 0;
    for (int64_t i = 0; i < len && live; ++i) {
        memset(nxt, 0, sizeof(uint64_t) * words);
        for (int32_t w = 0; w < words; ++w) {
            uint64_t bits = cur[w];
            while (bits) {
                int q = w * 64 + __builtin_ctzll(bits);
                bits &= bits - 1;
                if (q >= n) break;
                const uint64_t *f = follow + (size_t)q * words;
                for (int32_t v = 0; v < words; ++v) nxt[v] |= f[v];
            }
        }
        const uint64_t *m = sym + (size_t)text[i] * words;
        live = 0;
        for (int32_t w = 0; w < words; ++w) { cur[w] = nxt[w] & m[w]; live |= cur[w] != 0; }
    }
    memcpy(out, cur, sizeof(uint64_t) * words);
    free(cur); free(nxt);
    return live;
}
