/*
 * pasur_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct fp64 CPU reference for the exact round-by-round CFR solver of
 * "Solving Pasur Using GPU-Accelerated Counterfactual Regret Minimization" (arXiv 2508.06559).
 * Only the test suite, the smoke check and the benchmark's CPU-baseline / reference arm may load
 * this library.  It shares no code, header, table or constant generator with the CUDA library:
 * every rule below is restated here from the paper.
 *
 * Parity status per function (what pins each one is listed in the tests):
 *   or_splitmix64 / or_xoshiro / or_deal   pinned (published generator outputs, deal invariants)
 *   or_subsets_sum                         pinned (2764 sum-to-11 subsets, PyTorch section
 *                                          "Numerical Actions")
 *   or_legal_actions / or_apply /
 *   or_round_end / or_final_leaf           pinned (both worked games, Fig. game_0 / game_9)
 *   or_build_round / or_unfold             pinned (brute-force recursive count; Unfolding example)
 *   or_next_roots                          pinned (score normalisation example; invariants)
 *   or_cfr                                 pinned (T=1 closed form; minimax convergence; LP value;
 *                                          regret identity; zero-sum / delta invariance; every
 *                                          edge's R and S after T = 1, 2, 3 by hand on a two-ply
 *                                          game, vanilla and DCFR(1.5, 0, 2))
 *   or_minimax / or_best_response          pinned (scipy LP on tiny subgames; BR_B <= v <= BR_A)
 *   or_node_values                         pinned (level 0 equals or_root_values; every internal
 *                                          node is its children's max / min / sigma-mean)
 *   or_philox4x64                          pinned (numpy's Philox bit generator, a library routine)
 *   or_selfplay                            pinned (sample mean and outcome frequencies against the
 *                                          exact values below; pure strategies give one game)
 *   or_outcome_distribution                pinned (its mean equals the on-policy root value of
 *                                          or_root_values chained over the rounds; sums to 1)
 *
 * Conventions (the paper's, restated):
 *   card id = 4*rank + suit, rank 0 = Ace .. 9 = Ten, 10 = J, 11 = Q, 12 = K; suit 0 = clubs,
 *   1 = diamonds, 2 = hearts, 3 = spades (Fig. "Mapping Cards to Indices", Table card index sets).
 *   Player 0 = Alex (moves first every round), player 1 = Bob.  Utilities are Alex minus Bob.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define NUMERIC_MASK ((1ULL << 40) - 1ULL)
#define JACK_MASK (0xFULL << 40)
#define QUEEN_MASK (0xFULL << 44)
#define KING_MASK (0xFULL << 48)

/* ------------------------------------------------------------------------------------------ */
/* Generators (input side: the seeded deal).  SplitMix64 and xoshiro256** are written from    */
/* their published definitions (Steele/Lea/Flood 2014; Blackman/Vigna 2018); the bounded draw */
/* is Lemire's multiply-and-reject method (2019).                                              */
/* ------------------------------------------------------------------------------------------ */

static uint64_t splitmix_step(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xo_t;

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void xo_seed(xo_t *g, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; i++) g->s[i] = splitmix_step(&x);
}

static uint64_t xo_next(xo_t *g) {
    uint64_t *s = g->s;
    uint64_t result = rotl64(s[1] * 5ULL, 7) * 9ULL;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* uniform integer in [0, n) without modulo bias */
static uint64_t xo_below(xo_t *g, uint64_t n) {
    unsigned __int128 m = (unsigned __int128)xo_next(g) * n;
    uint64_t lo = (uint64_t)m;
    if (lo < n) {
        uint64_t thresh = (0ULL - n) % n;
        while (lo < thresh) {
            m = (unsigned __int128)xo_next(g) * n;
            lo = (uint64_t)m;
        }
    }
    return (uint64_t)(m >> 64);
}

void or_splitmix64(uint64_t seed, int n, uint64_t *out) {
    uint64_t x = seed;
    for (int i = 0; i < n; i++) out[i] = splitmix_step(&x);
}

void or_xoshiro(uint64_t seed, int n, uint64_t *out) {
    xo_t g;
    xo_seed(&g, seed);
    for (int i = 0; i < n; i++) out[i] = xo_next(&g);
}

/* xoshiro256** from a raw state (for the generator's published test values) */
void or_xoshiro_state(const uint64_t *s4, int n, uint64_t *out) {
    xo_t g;
    memcpy(g.s, s4, sizeof g.s);
    for (int i = 0; i < n; i++) out[i] = xo_next(&g);
}

/* uniform draws below n[i] (Lemire) from a seeded stream, for the bias test */
void or_below_seq(uint64_t seed, int count, const uint64_t *n, uint64_t *out) {
    xo_t g;
    xo_seed(&g, seed);
    for (int i = 0; i < count; i++) out[i] = xo_below(&g, n[i]);
}

static int is_jack(int c) { return c >= 40 && c < 44; }

/*
 * Seeded deal (§Pasur): shuffle 52 cards; deck[0:4] is the initial pool and may hold no Jack.
 * One Jack there is returned and replaced by the next card (swap with deck[4]); two or more
 * Jacks, or a replacement that is itself a Jack, force a reshuffle (a fresh Fisher-Yates of
 * 0..51 with the generator stream continued).  Round r deals deck[4+8r : 8+8r] to Alex and
 * deck[8+8r : 12+8r] to Bob.  Returns the number of shuffles used.
 */
int or_deal(uint64_t seed, uint8_t *deck) {
    xo_t g;
    xo_seed(&g, seed);
    for (int attempt = 1;; attempt++) {
        for (int i = 0; i < 52; i++) deck[i] = (uint8_t)i;
        for (int i = 51; i >= 1; i--) {
            int j = (int)xo_below(&g, (uint64_t)(i + 1));
            uint8_t t = deck[i];
            deck[i] = deck[j];
            deck[j] = t;
        }
        int nj = 0, pos = -1;
        for (int i = 0; i < 4; i++)
            if (is_jack(deck[i])) { nj++; pos = i; }
        if (nj == 0) return attempt;
        if (nj == 1 && !is_jack(deck[4])) {
            uint8_t t = deck[pos];
            deck[pos] = deck[4];
            deck[4] = t;
            return attempt;
        }
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Cards and rules (§Pasur, Table "Capture rules for each card type", Table "Pasur Scoring     */
/* System", Table card index sets).                                                            */
/* ------------------------------------------------------------------------------------------ */

static int card_value(int c) { return (c >> 2) + 1; }           /* numeric cards only: A=1..10 */
static int is_club(int c) { return (c & 3) == 0; }
static int card_points(int c) {
    if (c < 4) return 1;            /* each Ace */
    if (c == 4) return 2;           /* two of clubs */
    if (c == 37) return 3;          /* ten of diamonds */
    if (c >= 40 && c < 44) return 1;/* each Jack */
    return 0;
}
static int popcount64(uint64_t x) { int n = 0; while (x) { x &= x - 1; n++; } return n; }
static int clubs_in(uint64_t m) {
    int n = 0;
    for (int c = 0; c < 52; c += 4) n += (int)((m >> c) & 1ULL);
    return n;
}
static int points_in(uint64_t m) {
    int n = 0;
    for (int c = 0; c < 52; c++) if ((m >> c) & 1ULL) n += card_points(c);
    return n;
}

/* all subsets of the numeric cards in `avail` whose values sum to `target` (recursive
 * include/exclude over the cards in ascending id), written unsorted into out */
static void subsets_rec(const int *cards, int n, int i, int remaining, uint64_t cur,
                        uint64_t **out, int64_t *cnt, int64_t *cap) {
    if (remaining == 0 && cur != 0) {
        if (*cnt == *cap) {
            *cap = *cap ? *cap * 2 : 64;
            *out = (uint64_t *)realloc(*out, (size_t)*cap * sizeof(uint64_t));
        }
        (*out)[(*cnt)++] = cur;
        return;
    }
    if (i == n || remaining <= 0) return;
    int v = card_value(cards[i]);
    if (v <= remaining) subsets_rec(cards, n, i + 1, remaining - v, cur | (1ULL << cards[i]), out, cnt, cap);
    subsets_rec(cards, n, i + 1, remaining, cur, out, cnt, cap);
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Sorted list of nonempty subsets of the numeric cards of `avail` with value sum `target`.
 * Returns the count; writes up to cap masks. */
int64_t or_subsets_sum(uint64_t avail, int target, uint64_t *out, int64_t cap) {
    int cards[40], n = 0;
    for (int c = 0; c < 40; c++) if ((avail >> c) & 1ULL) cards[n++] = c;
    uint64_t *buf = NULL;
    int64_t cnt = 0, bcap = 0;
    subsets_rec(cards, n, 0, target, 0ULL, &buf, &cnt, &bcap);
    if (cnt > 1) qsort(buf, (size_t)cnt, sizeof(uint64_t), cmp_u64);
    for (int64_t i = 0; i < cnt && i < cap; i++) out[i] = buf[i];
    free(buf);
    return cnt;
}

/*
 * Legal actions of the player holding `hand` against `pool` (Table "Capture rules"):
 *   numeric card c: one action per nonempty subset P of the pool's numeric cards with
 *                   value(c) + sum(P) = 11; if there is none, c is laid (pick = 0).
 *                   The must-capture rule binds per card: other cards may still be laid.
 *   Jack:           one action picking every pool card that is not a King or Queen;
 *                   with nothing to pick it is a lay.
 *   Queen / King:   one action per Queen / King of the pool (a single card each);
 *                   with none, a lay.
 * Canonical order: lay card ascending, then pick mask ascending.
 * Returns the number of actions (writes at most cap).
 */
int or_legal_actions(uint64_t hand, uint64_t pool, int *lay, uint64_t *pick, int cap) {
    int n = 0;
    for (int c = 0; c < 52; c++) {
        if (!((hand >> c) & 1ULL)) continue;
        if (c < 40) {
            uint64_t tmp[4096];
            int64_t k = or_subsets_sum(pool & NUMERIC_MASK, 11 - card_value(c), tmp, 4096);
            if (k > 4096) k = 4096; /* cannot happen with 52 cards and target <= 10 */
            if (k == 0) {
                if (n < cap) { lay[n] = c; pick[n] = 0; }
                n++;
            }
            for (int64_t i = 0; i < k; i++) {
                if (n < cap) { lay[n] = c; pick[n] = tmp[i]; }
                n++;
            }
        } else if (c < 44) {
            uint64_t p = pool & (NUMERIC_MASK | JACK_MASK);
            if (n < cap) { lay[n] = c; pick[n] = p; }
            n++;
        } else {
            uint64_t same = pool & (c < 48 ? QUEEN_MASK : KING_MASK);
            if (same == 0) {
                if (n < cap) { lay[n] = c; pick[n] = 0; }
                n++;
            } else {
                for (int q = 0; q < 52; q++) {
                    if (!((same >> q) & 1ULL)) continue;
                    if (n < cap) { lay[n] = c; pick[n] = 1ULL << q; }
                    n++;
                }
            }
        }
    }
    return n;
}

/* Running score of a round (Table "Column definitions for the running-score tensor"):
 * rus[0] Alex clubs, [1] Bob clubs, [2] last picker (0 none, 1 Alex, 2 Bob), [3] Alex points,
 * [4] Alex surs, [5] Bob points, [6] Bob surs. */
typedef struct { uint64_t ha, hb, pool; int8_t rus[7]; } or_state;

/*
 * One move (CodeSnippet "ApplyActions" plus the running-score update the paper leaves out):
 * with an empty pick the card joins the pool; otherwise the card and the picked cards leave
 * the game into the mover's captures, adding their clubs and points, the mover becomes the
 * last picker, and clearing the pool is a Sur unless the card is a Jack or the round is the
 * final one.
 */
void or_apply(const uint64_t *in3, const int8_t *rus_in, int mover, int lay, uint64_t pick,
              int final_round, uint64_t *out3, int8_t *rus_out) {
    uint64_t h[2] = {in3[0], in3[1]}, pool = in3[2];
    int8_t r[7];
    memcpy(r, rus_in, 7);
    h[mover] &= ~(1ULL << lay);
    if (pick == 0) {
        pool |= 1ULL << lay;
    } else {
        pool &= ~pick;
        uint64_t cap = pick | (1ULL << lay);
        r[mover] = (int8_t)(r[mover] + clubs_in(cap));
        r[3 + 2 * mover] = (int8_t)(r[3 + 2 * mover] + points_in(cap));
        r[2] = (int8_t)(mover + 1);
        if (pool == 0 && !is_jack(lay) && !final_round) r[4 + 2 * mover] += 1;
    }
    out3[0] = h[0];
    out3[1] = h[1];
    out3[2] = pool;
    memcpy(rus_out, r, 7);
}

/* Points Alex minus Bob earned in a round: points plus 5 per Sur (Table "Pasur Scoring"). */
static int round_diff(const int8_t *r) { return (r[3] + 5 * r[4]) - (r[5] + 5 * r[6]); }

/*
 * Score carried between rounds (Table "Column definitions for the score tensor"):
 * (Alex clubs, Bob clubs, point difference, 7-clubs bonus), bonus 0 none / 1 Alex / 2 Bob.
 * Normalisation (§Score Tensors): once a player holds at least 7 clubs the bonus is recorded
 * and both club counts are reset to 0 and no longer tracked ([3,8,2,0] -> [0,0,2,2]).
 */
void or_normalize_score(int16_t *s) {
    if (s[3] == 0) {
        if (s[0] >= 7) { s[0] = 0; s[1] = 0; s[3] = 1; }
        else if (s[1] >= 7) { s[0] = 0; s[1] = 0; s[3] = 2; }
    } else {
        s[0] = 0;
        s[1] = 0;
    }
}

/* End of a non-final round: inherited score + this round's clubs and point difference. */
void or_round_end(const int16_t *score_in, const int8_t *rus, int16_t *score_out) {
    score_out[0] = (int16_t)(score_in[0] + rus[0]);
    score_out[1] = (int16_t)(score_in[1] + rus[1]);
    score_out[2] = (int16_t)(score_in[2] + round_diff(rus));
    score_out[3] = score_in[3];
    or_normalize_score(score_out);
}

/*
 * Leaf of the final round.  CleanUp (caption of Fig. game_0): the last picker takes what is
 * left in the pool, with its clubs and points; if nobody picked in the final round the pool is
 * discarded.  The value-to-go of the leaf is this round's difference plus the 7-clubs bonus,
 * +7 for Alex, -7 for Bob, 0 if nobody reached 7 (eq. final_util and eq. passuputil).
 * Writes the final normalised score when score_out is non-NULL.
 */
double or_final_leaf(const int16_t *score_in, const int8_t *rus_in, uint64_t pool, int16_t *score_out) {
    int8_t r[7];
    memcpy(r, rus_in, 7);
    if (r[2] != 0 && pool != 0) {
        int w = r[2] - 1;
        r[w] = (int8_t)(r[w] + clubs_in(pool));
        r[3 + 2 * w] = (int8_t)(r[3 + 2 * w] + points_in(pool));
    }
    int16_t s[4];
    or_round_end(score_in, r, s);
    if (score_out) memcpy(score_out, s, sizeof s);
    double bonus = s[3] == 1 ? 7.0 : (s[3] == 2 ? -7.0 : 0.0);
    return (double)round_diff(r) + bonus;
}

/* ------------------------------------------------------------------------------------------ */
/* Round game tree (GT) in level order, and its unfolding into the full game tree (FGT).      */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int round, final_round;
    uint8_t deck[52];
    int64_t n[9];
    int64_t *parent[9];      /* index in level k-1 (level 0: -1) */
    int64_t *child_beg[9];   /* first child in level k+1 */
    int32_t *nchild[9];
    int32_t *lay[9];         /* card played on the edge into this node (-1 at roots) */
    uint64_t *pick[9];
    uint64_t *st[9];         /* 3 masks per node: Alex hand, Bob hand, pool */
    int8_t *rus[9];          /* 7 per node */
    int64_t *root_of[9];
    /* FGT */
    int unfolded;
    int64_t n_roots;
    int64_t *score_off;      /* per GT root, n_roots+1 */
    int16_t *scores;         /* 4 per score slot */
    int64_t *fgt_off[9];     /* per level, n[k]+1: first FGT node of each GT node */
    int64_t nq[9];
} or_tree;

static uint64_t hand_mask(const uint8_t *deck, int lo) {
    uint64_t m = 0;
    for (int i = lo; i < lo + 4; i++) m |= 1ULL << deck[i];
    return m;
}

/*
 * Level-ordered GT of round `round` for the given root pools (§Game Tensor, §Actions): level 0
 * holds the roots in the given order; level k+1 holds the children of level k's nodes,
 * concatenated in parent order, each node's children in canonical action order.  Alex moves
 * at even plies, Bob at odd plies; every path has exactly 8 moves.
 */
or_tree *or_build_round(const uint8_t *deck, int round, const uint64_t *root_pools, int64_t n_roots) {
    if (round < 0 || round > 5 || n_roots < 0) return NULL;
    or_tree *t = (or_tree *)calloc(1, sizeof(or_tree));
    t->round = round;
    t->final_round = (round == 5);
    memcpy(t->deck, deck, 52);
    uint64_t ha = hand_mask(deck, 4 + 8 * round), hb = hand_mask(deck, 8 + 8 * round);
    t->n[0] = n_roots;
    t->parent[0] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_roots + 1));
    t->lay[0] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_roots + 1));
    t->pick[0] = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n_roots + 1));
    t->st[0] = (uint64_t *)malloc(sizeof(uint64_t) * 3 * (size_t)(n_roots + 1));
    t->rus[0] = (int8_t *)calloc((size_t)(n_roots + 1) * 7, 1);
    t->root_of[0] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_roots + 1));
    for (int64_t i = 0; i < n_roots; i++) {
        t->parent[0][i] = -1;
        t->lay[0][i] = -1;
        t->pick[0][i] = 0;
        t->st[0][3 * i] = ha;
        t->st[0][3 * i + 1] = hb;
        t->st[0][3 * i + 2] = root_pools[i];
        t->root_of[0][i] = i;
    }
    for (int k = 0; k < 8; k++) {
        int mover = k & 1;
        int64_t m = t->n[k];
        t->child_beg[k] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
        t->nchild[k] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
        int64_t total = 0;
        int lay[4096];
        uint64_t pick[4096];
        for (int64_t i = 0; i < m; i++) {
            uint64_t *s = &t->st[k][3 * i];
            int d = or_legal_actions(s[mover], s[2], lay, pick, 4096);
            t->child_beg[k][i] = total;
            t->nchild[k][i] = d;
            total += d;
        }
        t->child_beg[k][m] = total;
        int kk = k + 1;
        t->n[kk] = total;
        size_t cap = (size_t)total + 1;
        t->parent[kk] = (int64_t *)malloc(sizeof(int64_t) * cap);
        t->lay[kk] = (int32_t *)malloc(sizeof(int32_t) * cap);
        t->pick[kk] = (uint64_t *)malloc(sizeof(uint64_t) * cap);
        t->st[kk] = (uint64_t *)malloc(sizeof(uint64_t) * 3 * cap);
        t->rus[kk] = (int8_t *)malloc(7 * cap);
        t->root_of[kk] = (int64_t *)malloc(sizeof(int64_t) * cap);
        for (int64_t i = 0; i < m; i++) {
            uint64_t *s = &t->st[k][3 * i];
            int d = or_legal_actions(s[mover], s[2], lay, pick, 4096);
            for (int a = 0; a < d; a++) {
                int64_t c = t->child_beg[k][i] + a;
                t->parent[kk][c] = i;
                t->lay[kk][c] = lay[a];
                t->pick[kk][c] = pick[a];
                t->root_of[kk][c] = t->root_of[k][i];
                or_apply(s, &t->rus[k][7 * i], mover, lay[a], pick[a], t->final_round,
                         &t->st[kk][3 * c], &t->rus[kk][7 * c]);
            }
        }
    }
    return t;
}

void or_tree_free(or_tree *t) {
    if (!t) return;
    for (int k = 0; k < 9; k++) {
        free(t->parent[k]); free(t->child_beg[k]); free(t->nchild[k]); free(t->lay[k]);
        free(t->pick[k]); free(t->st[k]); free(t->rus[k]); free(t->root_of[k]); free(t->fgt_off[k]);
    }
    free(t->score_off);
    free(t->scores);
    free(t);
}

void or_tree_sizes(const or_tree *t, int64_t *n9, int64_t *nq9) {
    for (int k = 0; k < 9; k++) {
        if (n9) n9[k] = t->n[k];
        if (nq9) nq9[k] = t->unfolded ? t->nq[k] : -1;
    }
}

/* Export one GT level: any output may be NULL. */
void or_tree_level(const or_tree *t, int k, int64_t *parent, int32_t *nchild, int32_t *lay,
                   uint64_t *pick, uint64_t *state3, int8_t *rus7, int64_t *root_of) {
    int64_t m = t->n[k];
    for (int64_t i = 0; i < m; i++) {
        if (parent) parent[i] = t->parent[k][i];
        if (nchild) nchild[i] = k < 8 ? t->nchild[k][i] : 0;
        if (lay) lay[i] = t->lay[k][i];
        if (pick) pick[i] = t->pick[k][i];
        if (state3) memcpy(&state3[3 * i], &t->st[k][3 * i], 3 * sizeof(uint64_t));
        if (rus7) memcpy(&rus7[7 * i], &t->rus[k][7 * i], 7);
        if (root_of) root_of[i] = t->root_of[k][i];
    }
}

/*
 * Unfolding Process (§In-Hand Updates, Fig. "Unfolding Process"): GT root g carries the score
 * slots score_off[g] .. score_off[g+1]-1; every GT node inherits its root's slots.  FGT level k
 * lists, for each GT node of level k in order, one node per slot (GT-major, slot-minor), so the
 * parent of FGT node (j, s) is (parent(j), s).  Returns 0 on success.
 */
int or_unfold(or_tree *t, const int64_t *score_off, const int16_t *scores, int64_t *nq_out) {
    int64_t R = t->n[0];
    free(t->score_off);
    free(t->scores);
    t->n_roots = R;
    t->score_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(R + 1));
    memcpy(t->score_off, score_off, sizeof(int64_t) * (size_t)(R + 1));
    int64_t ns = score_off[R];
    t->scores = (int16_t *)malloc(sizeof(int16_t) * 4 * (size_t)(ns + 1));
    memcpy(t->scores, scores, sizeof(int16_t) * 4 * (size_t)ns);
    for (int k = 0; k < 9; k++) {
        free(t->fgt_off[k]);
        t->fgt_off[k] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(t->n[k] + 1));
        int64_t acc = 0;
        for (int64_t j = 0; j < t->n[k]; j++) {
            t->fgt_off[k][j] = acc;
            int64_t g = t->root_of[k][j];
            acc += score_off[g + 1] - score_off[g];
        }
        t->fgt_off[k][t->n[k]] = acc;
        t->nq[k] = acc;
        if (nq_out) nq_out[k] = acc;
    }
    t->unfolded = 1;
    return 0;
}

/* FGT parent of every FGT node of level k (k >= 1): t_edg of the Unfolding Process. */
int or_fgt_parents(const or_tree *t, int k, int64_t *out) {
    if (!t->unfolded || k < 1 || k > 8) return -1;
    for (int64_t j = 0; j < t->n[k]; j++) {
        int64_t p = t->parent[k][j];
        int64_t S = t->fgt_off[k][j + 1] - t->fgt_off[k][j];
        for (int64_t s = 0; s < S; s++) out[t->fgt_off[k][j] + s] = t->fgt_off[k - 1][p] + s;
    }
    return 0;
}

static const int16_t *slot_score(const or_tree *t, int64_t gt_root, int64_t s) {
    return &t->scores[4 * (t->score_off[gt_root] + s)];
}

/* Leaf values of the final round for every FGT leaf (level 8), in FGT order. */
int or_leaf_utilities_final(const or_tree *t, double *out) {
    if (!t->unfolded || !t->final_round) return -1;
    for (int64_t j = 0; j < t->n[8]; j++) {
        int64_t g = t->root_of[8][j];
        int64_t S = t->fgt_off[8][j + 1] - t->fgt_off[8][j];
        for (int64_t s = 0; s < S; s++)
            out[t->fgt_off[8][j] + s] = or_final_leaf(slot_score(t, g, s), &t->rus[8][7 * j],
                                                      t->st[8][3 * j + 2], NULL);
    }
    return 0;
}

/* ---- next-round roots (§Between-Hand Updates, CodeSnippet "BetweenHands") ---- */

typedef struct { uint64_t pool; int16_t s[4]; int64_t leaf; } nr_item;

static int cmp_nr(const void *a, const void *b) {
    const nr_item *x = (const nr_item *)a, *y = (const nr_item *)b;
    if (x->pool != y->pool) return x->pool < y->pool ? -1 : 1;
    for (int i = 0; i < 4; i++)
        if (x->s[i] != y->s[i]) return x->s[i] < y->s[i] ? -1 : 1;
    return x->leaf < y->leaf ? -1 : (x->leaf > y->leaf ? 1 : 0);
}

/*
 * The next round's FGT roots: for every FGT leaf (j, s) the next root is (pool at j,
 * normalise(score s + running score of j)).  Roots are the unique pools in ascending order and,
 * per pool, the unique scores in lexicographic (Alex clubs, Bob clubs, difference, bonus)
 * order.  lnk[leaf] = index of the leaf's next FGT root (t_lnk).  Outputs may be NULL (query).
 * Returns the number of next FGT roots; *n_pools gets the number of distinct pools.
 */
int64_t or_next_roots(const or_tree *t, uint64_t *pools_out, int64_t *score_off_out,
                      int16_t *scores_out, int64_t *lnk_out, int64_t *n_pools) {
    if (!t->unfolded || t->final_round) return -1;
    int64_t Q = t->nq[8];
    nr_item *it = (nr_item *)malloc(sizeof(nr_item) * (size_t)(Q + 1));
    for (int64_t j = 0; j < t->n[8]; j++) {
        int64_t g = t->root_of[8][j];
        int64_t S = t->fgt_off[8][j + 1] - t->fgt_off[8][j];
        for (int64_t s = 0; s < S; s++) {
            int64_t q = t->fgt_off[8][j] + s;
            it[q].pool = t->st[8][3 * j + 2];
            or_round_end(slot_score(t, g, s), &t->rus[8][7 * j], it[q].s);
            it[q].leaf = q;
        }
    }
    qsort(it, (size_t)Q, sizeof(nr_item), cmp_nr);
    int64_t nroot = -1, npool = -1;
    for (int64_t i = 0; i < Q; i++) {
        int new_pool = (i == 0) || it[i].pool != it[i - 1].pool;
        int new_root = new_pool || memcmp(it[i].s, it[i - 1].s, sizeof it[i].s) != 0;
        if (new_pool) {
            npool++;
            if (pools_out) pools_out[npool] = it[i].pool;
            if (score_off_out) score_off_out[npool] = nroot + 1;
        }
        if (new_root) {
            nroot++;
            if (scores_out) memcpy(&scores_out[4 * nroot], it[i].s, sizeof it[i].s);
        }
        if (lnk_out) lnk_out[it[i].leaf] = nroot;
    }
    nroot++;
    npool++;
    if (score_off_out) score_off_out[npool] = nroot;
    if (n_pools) *n_pools = npool;
    free(it);
    return nroot;
}

/* Leaf values of a non-final round (eq. passuputil): this round's point difference plus the
 * next round's root value at the linked root. */
int or_leaf_utilities_linked(const or_tree *t, const int64_t *lnk, const double *u_next, double *out) {
    if (!t->unfolded) return -1;
    for (int64_t j = 0; j < t->n[8]; j++) {
        int64_t S = t->fgt_off[8][j + 1] - t->fgt_off[8][j];
        int d = round_diff(&t->rus[8][7 * j]);
        for (int64_t s = 0; s < S; s++) {
            int64_t q = t->fgt_off[8][j] + s;
            out[q] = (double)d + u_next[lnk[q]];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* CFR (§CFR Algorithm; eq. RM, eq. avsigma; DCFR eqs. DFCR_REG / DFCR_AVG).                   */
/* Every FGT node is its own information set (open hands).                                     */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    const or_tree *t;
    const double *leaf;
    double *R[9], *S[9];     /* per FGT edge, levels 1..8 */
    int it;                  /* current iteration t = 1..T */
    double thresh;           /* RM dead zone for this iteration */
    int variant;             /* 0 vanilla, 1 DCFR */
    double alpha, beta, gamma;
} cfr_ctx;

/* regret matching: sigma proportional to the positive part of the cumulative regrets (eq. RM);
 * regrets not above the dead zone count as zero; uniform when no regret is positive */
static void regret_match(const double *R, int d, double thr, double *sig) {
    double sum = 0.0;
    for (int a = 0; a < d; a++) sum += R[a] > thr ? R[a] : 0.0;
    for (int a = 0; a < d; a++) sig[a] = sum > 0.0 ? (R[a] > thr ? R[a] : 0.0) / sum : 1.0 / d;
}

static double cfr_rec(cfr_ctx *c, int k, int64_t j, int64_t s, double pi0, double pi1) {
    const or_tree *t = c->t;
    if (k == 8) return c->leaf[t->fgt_off[8][j] + s];
    int d = t->nchild[k][j];
    int p = k & 1;
    double sp = p == 0 ? 1.0 : -1.0;
    int64_t cb = t->child_beg[k][j];
    double *sig = (double *)malloc(sizeof(double) * (size_t)d * 3);
    double *Rloc = sig + d, *vch = sig + 2 * d;
    for (int a = 0; a < d; a++) Rloc[a] = c->R[k + 1][t->fgt_off[k + 1][cb + a] + s];
    regret_match(Rloc, d, c->thresh, sig);
    for (int a = 0; a < d; a++) {
        double n0 = pi0, n1 = pi1;
        if (p == 0) n0 *= sig[a]; else n1 *= sig[a];
        vch[a] = cfr_rec(c, k + 1, cb + a, s, n0, n1);
    }
    double v = vch[0];
    for (int a = 0; a < d; a++) v += sig[a] * (vch[a] - vch[0]);
    double pi_p = p == 0 ? pi0 : pi1, pi_o = p == 0 ? pi1 : pi0;
    for (int a = 0; a < d; a++) {
        int64_t q = t->fgt_off[k + 1][cb + a] + s;
        double r = sp * pi_o * (vch[a] - v);
        if (c->variant == 1) {
            /* DCFR: discount the previous cumulative regret by t'^a/(t'^a+1) (positive) or
             * t'^b/(t'^b+1) (otherwise) with t' = t-1, then add the instant regret */
            double tp = (double)(c->it - 1);
            double Rold = c->R[k + 1][q];
            double f = Rold > 0.0 ? pow(tp, c->alpha) / (pow(tp, c->alpha) + 1.0)
                                  : pow(tp, c->beta) / (pow(tp, c->beta) + 1.0);
            c->R[k + 1][q] = Rold * f + r;
            double g = c->it > 1 ? pow(1.0 - 1.0 / (double)c->it, c->gamma) : 0.0;
            c->S[k + 1][q] = c->S[k + 1][q] * g + pi_p * sig[a];
        } else {
            c->R[k + 1][q] += r;
            c->S[k + 1][q] += pi_p * sig[a];
        }
    }
    free(sig);
    return v;
}

/* Umax of every FGT root: the largest |leaf value| in its own subtree (the dead-zone scale of
 * regret matching, so that each root's solve depends on its subtree alone). */
static double *root_umax(const or_tree *t, const double *leaf) {
    double *um = (double *)calloc((size_t)t->nq[0] + 1, sizeof(double));
    for (int64_t j = 0; j < t->n[8]; j++) {
        int64_t g = t->root_of[8][j];
        int64_t S = t->fgt_off[8][j + 1] - t->fgt_off[8][j];
        for (int64_t s = 0; s < S; s++) {
            double a = fabs(leaf[t->fgt_off[8][j] + s]);
            int64_t q = t->fgt_off[0][g] + s;
            if (a > um[q]) um[q] = a;
        }
    }
    return um;
}

/*
 * T iterations of CFR on an unfolded round with the given FGT leaf values (eq. final_util /
 * eq. passuputil), simultaneous updates, root reach 1 for both players.  Iteration t:
 * sigma^t from the regrets by regret matching with dead zone tau*t*Umax (Umax = max |leaf| over the
 * FGT root's own subtree);
 * reach top-down; values bottom-up v(h) = v(a0) + sum_a sigma(a) (v(h.a) - v(a0));
 * R(h,a) += s_p pi_{-p}(h) (v(h.a) - v(h)), S(h,a) += pi_p(h) sigma(h,a);  Uacc(root) += v(root).
 * Outputs (any may be NULL): sigma_bar per FGT edge by level (levels 1..8 concatenated, i.e.
 * index fgt level-1 offset + q; normalised S, uniform where sum S = 0), U per FGT root =
 * Uacc/T (the average root utility of CodeSnippet "CFR"), and the final R and S.
 * variant 0 = vanilla CFR, 1 = DCFR(alpha, beta, gamma).
 */
int or_cfr(const or_tree *t, const double *leaf, int iters, double tau, int variant,
           double alpha, double beta, double gamma, double *sigma_bar, double *U, double *R_out,
           double *S_out) {
    if (!t->unfolded || iters < 0) return -1;
    cfr_ctx c;
    memset(&c, 0, sizeof c);
    c.t = t;
    c.leaf = leaf;
    c.variant = variant;
    c.alpha = alpha; c.beta = beta; c.gamma = gamma;
    for (int k = 1; k <= 8; k++) {
        c.R[k] = (double *)calloc((size_t)t->nq[k] + 1, sizeof(double));
        c.S[k] = (double *)calloc((size_t)t->nq[k] + 1, sizeof(double));
    }
    double *umax = root_umax(t, leaf);
    double *uacc = (double *)calloc((size_t)t->nq[0] + 1, sizeof(double));
    for (int it = 1; it <= iters; it++) {
        c.it = it;
        for (int64_t j = 0; j < t->n[0]; j++) {
            int64_t S = t->fgt_off[0][j + 1] - t->fgt_off[0][j];
            for (int64_t s = 0; s < S; s++) {
                int64_t q = t->fgt_off[0][j] + s;
                c.thresh = tau * (double)it * umax[q];
                uacc[q] += cfr_rec(&c, 0, j, s, 1.0, 1.0);
            }
        }
    }
    free(umax);
    if (U)
        for (int64_t q = 0; q < t->nq[0]; q++) U[q] = iters > 0 ? uacc[q] / iters : 0.0;
    int64_t base = 0;
    for (int k = 1; k <= 8; k++) {
        if (sigma_bar) {
            for (int64_t j = 0; j < t->n[k - 1]; j++) {
                int d = t->nchild[k - 1][j];
                int64_t cb = t->child_beg[k - 1][j];
                int64_t S = t->fgt_off[k - 1][j + 1] - t->fgt_off[k - 1][j];
                for (int64_t s = 0; s < S; s++) {
                    double sum = 0.0;
                    for (int a = 0; a < d; a++) sum += c.S[k][t->fgt_off[k][cb + a] + s];
                    for (int a = 0; a < d; a++) {
                        int64_t q = t->fgt_off[k][cb + a] + s;
                        sigma_bar[base + q] = sum > 0.0 ? c.S[k][q] / sum : 1.0 / d;
                    }
                }
            }
        }
        if (R_out) memcpy(R_out + base, c.R[k], sizeof(double) * (size_t)t->nq[k]);
        if (S_out) memcpy(S_out + base, c.S[k], sizeof(double) * (size_t)t->nq[k]);
        base += t->nq[k];
        free(c.R[k]);
        free(c.S[k]);
    }
    free(uacc);
    return 0;
}

/*
 * The same vanilla CFR carried out in float32 arithmetic (the precision of the paper's strategy
 * tensors, t_sgm float32).  Used only as a conditioning probe by the tests: an edge whose average
 * strategy differs between this run and the fp64 run is one whose value f32 rounding decides.
 */
typedef struct {
    const or_tree *t;
    const double *leaf;
    float *R[9], *S[9];
    float thresh;
} cfr32_ctx;

static float cfr32_rec(cfr32_ctx *c, int k, int64_t j, int64_t s, float pi0, float pi1) {
    const or_tree *t = c->t;
    if (k == 8) return (float)c->leaf[t->fgt_off[8][j] + s];
    int d = t->nchild[k][j];
    int p = k & 1;
    int64_t cb = t->child_beg[k][j];
    float *sig = (float *)malloc(sizeof(float) * (size_t)d * 2);
    float *vch = sig + d;
    float sum = 0.f;
    for (int a = 0; a < d; a++) {
        float r = c->R[k + 1][t->fgt_off[k + 1][cb + a] + s];
        sum += r > c->thresh ? r : 0.f;
    }
    for (int a = 0; a < d; a++) {
        float r = c->R[k + 1][t->fgt_off[k + 1][cb + a] + s];
        sig[a] = sum > 0.f ? (r > c->thresh ? r / sum : 0.f) : 1.f / (float)d;
    }
    for (int a = 0; a < d; a++)
        vch[a] = cfr32_rec(c, k + 1, cb + a, s, p == 0 ? pi0 * sig[a] : pi0, p == 0 ? pi1 : pi1 * sig[a]);
    float v = vch[0];
    for (int a = 0; a < d; a++) v += sig[a] * (vch[a] - vch[0]);
    float pi_p = p == 0 ? pi0 : pi1, pi_o = p == 0 ? pi1 : pi0, sp = p == 0 ? 1.f : -1.f;
    for (int a = 0; a < d; a++) {
        int64_t q = t->fgt_off[k + 1][cb + a] + s;
        c->R[k + 1][q] += sp * pi_o * (vch[a] - v);
        c->S[k + 1][q] += pi_p * sig[a];
    }
    free(sig);
    return v;
}

int or_cfr_f32(const or_tree *t, const double *leaf, int iters, double tau, double *sigma_bar, double *U) {
    if (!t->unfolded || iters < 0) return -1;
    cfr32_ctx c;
    memset(&c, 0, sizeof c);
    c.t = t;
    c.leaf = leaf;
    for (int k = 1; k <= 8; k++) {
        c.R[k] = (float *)calloc((size_t)t->nq[k] + 1, sizeof(float));
        c.S[k] = (float *)calloc((size_t)t->nq[k] + 1, sizeof(float));
    }
    double *umax = root_umax(t, leaf);
    double *uacc = (double *)calloc((size_t)t->nq[0] + 1, sizeof(double));
    for (int it = 1; it <= iters; it++) {
        for (int64_t j = 0; j < t->n[0]; j++) {
            int64_t S = t->fgt_off[0][j + 1] - t->fgt_off[0][j];
            for (int64_t s = 0; s < S; s++) {
                int64_t q = t->fgt_off[0][j] + s;
                c.thresh = (float)(tau * umax[q]) * (float)it;
                uacc[q] += cfr32_rec(&c, 0, j, s, 1.f, 1.f);
            }
        }
    }
    free(umax);
    if (U)
        for (int64_t q = 0; q < t->nq[0]; q++) U[q] = iters > 0 ? uacc[q] / iters : 0.0;
    int64_t base = 0;
    for (int k = 1; k <= 8; k++) {
        if (sigma_bar)
            for (int64_t j = 0; j < t->n[k - 1]; j++) {
                int d = t->nchild[k - 1][j];
                int64_t cb = t->child_beg[k - 1][j];
                int64_t S = t->fgt_off[k - 1][j + 1] - t->fgt_off[k - 1][j];
                for (int64_t s = 0; s < S; s++) {
                    double sum = 0.0;
                    for (int a = 0; a < d; a++) sum += c.S[k][t->fgt_off[k][cb + a] + s];
                    for (int a = 0; a < d; a++) {
                        int64_t q = t->fgt_off[k][cb + a] + s;
                        sigma_bar[base + q] = sum > 0.0 ? c.S[k][q] / sum : 1.0 / d;
                    }
                }
            }
        base += t->nq[k];
        free(c.R[k]);
        free(c.S[k]);
    }
    free(uacc);
    return 0;
}

/* ---- game values under fixed or optimal play ---- */

/* mode 0: minimax (Alex max, Bob min); 1: Alex best response to sigma (Bob follows sigma);
 * 2: Bob best response (Alex follows sigma); 3: both follow sigma; 4: both uniform */
static double value_rec(const or_tree *t, const double *leaf, const double *sig_lvl[9], int mode,
                        int k, int64_t j, int64_t s) {
    if (k == 8) return leaf[t->fgt_off[8][j] + s];
    int d = t->nchild[k][j];
    int p = k & 1;
    int64_t cb = t->child_beg[k][j];
    double best = 0.0, ev = 0.0;
    for (int a = 0; a < d; a++) {
        double v = value_rec(t, leaf, sig_lvl, mode, k + 1, cb + a, s);
        if (a == 0 || (p == 0 ? v > best : v < best)) best = v;
        double w = mode == 4 ? 1.0 / d : (sig_lvl[k + 1] ? sig_lvl[k + 1][t->fgt_off[k + 1][cb + a] + s] : 0.0);
        ev += w * v;
    }
    switch (mode) {
        case 0: return best;
        case 1: return p == 0 ? best : ev;
        case 2: return p == 1 ? best : ev;
        default: return ev;
    }
}

/* Value of every FGT root under `mode` (see value_rec); sigma is laid out like or_cfr's
 * sigma_bar output (may be NULL for modes 0 and 4). */
int or_root_values(const or_tree *t, const double *leaf, const double *sigma, int mode, double *out) {
    if (!t->unfolded) return -1;
    const double *sig_lvl[9] = {0};
    if (sigma) {
        int64_t base = 0;
        for (int k = 1; k <= 8; k++) {
            sig_lvl[k] = sigma + base;
            base += t->nq[k];
        }
    }
    for (int64_t j = 0; j < t->n[0]; j++) {
        int64_t S = t->fgt_off[0][j + 1] - t->fgt_off[0][j];
        for (int64_t s = 0; s < S; s++) out[t->fgt_off[0][j] + s] = value_rec(t, leaf, sig_lvl, mode, 0, j, s);
    }
    return 0;
}

/* Value of every FGT node under `mode` (see value_rec), levels 0..8 concatenated in FGT order
 * (out has sum of the 9 level sizes entries): the same recursion as or_root_values, keeping each
 * node's value.  Used by the tests to weigh a strategy difference at one node by the values of
 * its children. */
static double node_value_rec(const or_tree *t, const double *leaf, const double *sig_lvl[9], int mode, int k,
                             int64_t j, int64_t s, double *const out_lvl[9]) {
    double v;
    if (k == 8) {
        v = leaf[t->fgt_off[8][j] + s];
    } else {
        int d = t->nchild[k][j];
        int p = k & 1;
        int64_t cb = t->child_beg[k][j];
        double best = 0.0, ev = 0.0;
        for (int a = 0; a < d; a++) {
            double c = node_value_rec(t, leaf, sig_lvl, mode, k + 1, cb + a, s, out_lvl);
            if (a == 0 || (p == 0 ? c > best : c < best)) best = c;
            double w = mode == 4 ? 1.0 / d : (sig_lvl[k + 1] ? sig_lvl[k + 1][t->fgt_off[k + 1][cb + a] + s] : 0.0);
            ev += w * c;
        }
        v = mode == 0 ? best : mode == 1 ? (p == 0 ? best : ev) : mode == 2 ? (p == 1 ? best : ev) : ev;
    }
    out_lvl[k][t->fgt_off[k][j] + s] = v;
    return v;
}

int or_node_values(const or_tree *t, const double *leaf, const double *sigma, int mode, double *out) {
    if (!t->unfolded) return -1;
    const double *sig_lvl[9] = {0};
    double *out_lvl[9];
    int64_t base = 0, sbase = 0;
    for (int k = 0; k <= 8; k++) {
        out_lvl[k] = out + base;
        base += t->nq[k];
        if (k >= 1 && sigma) {
            sig_lvl[k] = sigma + sbase;
            sbase += t->nq[k];
        }
    }
    for (int64_t j = 0; j < t->n[0]; j++) {
        int64_t S = t->fgt_off[0][j + 1] - t->fgt_off[0][j];
        for (int64_t s = 0; s < S; s++) node_value_rec(t, leaf, sig_lvl, mode, 0, j, s, out_lvl);
    }
    return 0;
}

/* Brute-force count of the GT nodes of every level below one root by plain recursion over the
 * legal moves (no level lists): an independent check of or_build_round's level sizes. */
static void count_rec(uint64_t st[3], int8_t rus[7], int k, int final_round, int64_t *cnt) {
    cnt[k]++;
    if (k == 8) return;
    int lay[4096];
    uint64_t pick[4096];
    int mover = k & 1;
    int d = or_legal_actions(st[mover], st[2], lay, pick, 4096);
    for (int a = 0; a < d; a++) {
        uint64_t ns[3];
        int8_t nr[7];
        or_apply(st, rus, mover, lay[a], pick[a], final_round, ns, nr);
        count_rec(ns, nr, k + 1, final_round, cnt);
    }
}

void or_count_round(const uint8_t *deck, int round, uint64_t root_pool, int64_t *cnt9) {
    uint64_t st[3] = {hand_mask(deck, 4 + 8 * round), hand_mask(deck, 8 + 8 * round), root_pool};
    int8_t rus[7] = {0};
    for (int k = 0; k < 9; k++) cnt9[k] = 0;
    count_rec(st, rus, 0, round == 5, cnt9);
}

int or_popcount64(uint64_t x) { return popcount64(x); }

/*
 * Game value by plain backward induction over the rounds round..5 from one state, with no level
 * lists, score slots or links: at the end of a non-final round the score is carried
 * (or_round_end) and the next round starts from the pool with the next hands.  Returns the
 * value-to-go (Alex minus Bob points still to come, bonus included): an independent check of
 * the round-by-round chaining (eq. passuputil, CodeSnippet "BetweenHands").
 */
static double mm_rec(const uint8_t *deck, int round, uint64_t st[3], int8_t rus[7], const int16_t *score, int k) {
    if (k == 8) {
        if (round == 5) return or_final_leaf(score, rus, st[2], NULL);
        int16_t ns[4];
        or_round_end(score, rus, ns);
        uint64_t nst[3] = {hand_mask(deck, 4 + 8 * (round + 1)), hand_mask(deck, 8 + 8 * (round + 1)), st[2]};
        int8_t nr[7] = {0};
        return (double)round_diff(rus) + mm_rec(deck, round + 1, nst, nr, ns, 0);
    }
    int lay[4096];
    uint64_t pick[4096];
    int mover = k & 1;
    int d = or_legal_actions(st[mover], st[2], lay, pick, 4096);
    double best = 0.0;
    for (int a = 0; a < d; a++) {
        uint64_t ns[3];
        int8_t nr[7];
        or_apply(st, rus, mover, lay[a], pick[a], round == 5, ns, nr);
        double v = mm_rec(deck, round, ns, nr, score, k + 1);
        if (a == 0 || (mover == 0 ? v > best : v < best)) best = v;
    }
    return best;
}

double or_minimax_rounds(const uint8_t *deck, int round, uint64_t pool, const int16_t *score) {
    uint64_t st[3] = {hand_mask(deck, 4 + 8 * round), hand_mask(deck, 8 + 8 * round), pool};
    int8_t rus[7] = {0};
    return mm_rec(deck, round, st, rus, score, 0);
}

/* ------------------------------------------------------------------------------------------ */
/* Self-play (the fair-value simulation of the paper's introduction and its learned-strategy   */
/* study): games played from one FGT root through consecutive rounds, every move drawn from    */
/* the average strategy of the node reached, one choice per parent as in §External Sampling.   */
/* ------------------------------------------------------------------------------------------ */

/*
 * Philox4x64-10, written from its published definition (Salmon, Moraes, Dror and Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC 2011): ten rounds of two 64x64->128-bit
 * multiplications by fixed odd constants, the high halves xored with the other two counter
 * words and the round key, the key bumped by the two Weyl constants between rounds.
 */
void or_philox4x64(const uint64_t *ctr, const uint64_t *key, uint64_t *out) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        unsigned __int128 p0 = (unsigned __int128)M0 * x0, p1 = (unsigned __int128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The uniform draw of ply `ply` of game `game`: word 0 of Philox4x64-10 at counter
 * (ply, game, 0, 0) under key (seed, 0), its top 24 bits as a float in [0, 1). */
static float sp_uniform(uint64_t seed, int64_t game, int64_t ply) {
    uint64_t ctr[4] = {(uint64_t)ply, (uint64_t)game, 0, 0}, key[2] = {seed, 0}, o[4];
    or_philox4x64(ctr, key, o);
    return (float)(o[0] >> 40) * (1.0f / 16777216.0f);
}

/* Index of the GT root that owns FGT root q (fgt_off[0] is ascending). */
static int64_t gt_root_of(const or_tree *t, int64_t q) {
    int64_t lo = 0, hi = t->n[0] - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if (t->fgt_off[0][mid] <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* The final game difference at FGT leaf (j, s) of the final round: the score difference after
 * the round (inherited difference + the round's difference after CleanUp) plus the 7-clubs
 * bonus, +7 Alex / -7 Bob (eq. final_util). */
static int final_game_diff(const or_tree *t, int64_t j, int64_t s) {
    int16_t sc[4];
    or_final_leaf(slot_score(t, t->root_of[8][j], s), &t->rus[8][7 * j], t->st[8][3 * j + 2], sc);
    return sc[2] + (sc[3] == 1 ? 7 : (sc[3] == 2 ? -7 : 0));
}

/*
 * n_games games from FGT root root_q of rounds[0]; rounds[i+1] is the round after rounds[i],
 * lnk[i] its leaf-to-next-root links (or_next_roots), and the last round is the final one.
 * sigma[i]: float strategy of every FGT edge of rounds[i] (levels 1..8 concatenated, FGT order).
 * At every ply (numbered from 0 across the rounds) the mover's move is drawn as follows, in
 * float arithmetic: u = sp_uniform(seed, game, ply); with w_a the strategies of the node's
 * children in canonical order, total = w_0 + w_1 + ... (left to right) and target = u * total,
 * the move is the first a with w_0 + ... + w_a > target; when there is none (total 0 or a
 * rounding tie) it is the last a with w_a > 0, else a = 0.  out[g] = final game difference of
 * game g (Alex minus Bob points of the whole game including the root's inherited difference,
 * bonus included).  Returns 0, or -1 on invalid arguments.
 */
int or_selfplay(const or_tree *const *rounds, int n_rounds, const float *const *sigma, const int64_t *const *lnk,
                int64_t root_q, int64_t n_games, uint64_t seed, int16_t *out) {
    if (n_rounds < 1 || !rounds[n_rounds - 1]->final_round) return -1;
    for (int i = 0; i < n_rounds; i++)
        if (!rounds[i]->unfolded) return -1;
    if (root_q < 0 || root_q >= rounds[0]->nq[0]) return -1;
    for (int64_t g = 0; g < n_games; g++) {
        int64_t q = root_q, ply = 0;
        for (int i = 0; i < n_rounds; i++) {
            const or_tree *t = rounds[i];
            int64_t j = gt_root_of(t, q), s = q - t->fgt_off[0][j];
            int64_t base[9] = {0};
            for (int k = 2; k <= 8; k++) base[k] = base[k - 1] + t->nq[k - 1];
            for (int k = 0; k < 8; k++) {
                int d = t->nchild[k][j];
                int64_t cb = t->child_beg[k][j];
                float u = sp_uniform(seed, g, ply++);
                float total = 0.0f;
                for (int a = 0; a < d; a++) total += sigma[i][base[k + 1] + t->fgt_off[k + 1][cb + a] + s];
                float target = u * total, cum = 0.0f;
                int pick = -1, last_pos = -1;
                for (int a = 0; a < d; a++) {
                    float w = sigma[i][base[k + 1] + t->fgt_off[k + 1][cb + a] + s];
                    cum += w;
                    if (w > 0.0f) last_pos = a;
                    if (pick < 0 && cum > target) pick = a;
                }
                if (pick < 0) pick = last_pos >= 0 ? last_pos : 0;
                j = cb + pick;
            }
            int64_t leaf = t->fgt_off[8][j] + s;
            if (i + 1 < n_rounds) q = lnk[i][leaf];
            else out[g] = (int16_t)final_game_diff(t, j, s);
        }
    }
    return 0;
}

/*
 * Exact distribution of the final game difference when both players follow sigma (double,
 * laid out as in or_selfplay) from FGT root root_q: the probability of reaching every FGT node
 * is carried forward level by level (a child gets its parent's probability times its strategy),
 * each leaf's probability moves to its linked next-round root, and each final leaf adds its
 * probability to the bin of its final game difference.  prob[b] = P(difference = lo + b) for
 * b < n_bins.  Returns 0, or -1 on invalid arguments or a difference outside the bins.
 */
int or_outcome_distribution(const or_tree *const *rounds, int n_rounds, const double *const *sigma,
                            const int64_t *const *lnk, int64_t root_q, int lo, int n_bins, double *prob) {
    if (n_rounds < 1 || !rounds[n_rounds - 1]->final_round) return -1;
    for (int b = 0; b < n_bins; b++) prob[b] = 0.0;
    double *root_p = (double *)calloc((size_t)rounds[0]->nq[0] + 1, sizeof(double));
    root_p[root_q] = 1.0;
    int rc = 0;
    for (int i = 0; i < n_rounds && rc == 0; i++) {
        const or_tree *t = rounds[i];
        double *cur = root_p, *next = NULL;
        int64_t base = 0;
        for (int k = 0; k < 8; k++) {
            next = (double *)calloc((size_t)t->nq[k + 1] + 1, sizeof(double));
            for (int64_t j = 0; j < t->n[k]; j++) {
                int64_t S = t->fgt_off[k][j + 1] - t->fgt_off[k][j];
                for (int a = 0; a < t->nchild[k][j]; a++) {
                    int64_t c = t->child_beg[k][j] + a;
                    for (int64_t s = 0; s < S; s++) {
                        int64_t qc = t->fgt_off[k + 1][c] + s;
                        next[qc] = cur[t->fgt_off[k][j] + s] * sigma[i][base + qc];
                    }
                }
            }
            base += t->nq[k + 1];
            free(cur);
            cur = next;
        }
        if (i + 1 < n_rounds) {
            root_p = (double *)calloc((size_t)rounds[i + 1]->nq[0] + 1, sizeof(double));
            for (int64_t q = 0; q < t->nq[8]; q++) root_p[lnk[i][q]] += cur[q];
        } else {
            for (int64_t j = 0; j < t->n[8]; j++) {
                int64_t S = t->fgt_off[8][j + 1] - t->fgt_off[8][j];
                for (int64_t s = 0; s < S; s++) {
                    double p = cur[t->fgt_off[8][j] + s];
                    if (p == 0.0) continue;
                    int b = final_game_diff(t, j, s) - lo;
                    if (b < 0 || b >= n_bins) { rc = -1; break; }
                    prob[b] += p;
                }
                if (rc) break;
            }
        }
        free(cur);
    }
    return rc;
}
