/*
 * pasur.h -- C ABI of the GB300 (sm_103a) exact round-by-round CFR solver for two-player,
 * open-hand, fixed-deck Pasur, after "Solving Pasur Using GPU-Accelerated Counterfactual Regret
 * Minimization" (arXiv 2508.06559).
 *
 * General rules for every entry point
 *   - Every call returns a pasur_status (0 = PASUR_OK, negative = error).  The library throws
 *     no exception of its own; only a failed host-memory allocation inside a call (which the
 *     library does not recover from) could raise one.  After an error, pasur_last_error(ctx)
 *     holds a one-line message.
 *   - Pointers documented as "host or device" may point to host memory or to device memory of
 *     the context's device; the library detects which.  Device pointers are used on the
 *     context's stream; host results are complete when the call returns.
 *   - Caller-owned buffers are never retained after a call returns.
 *   - Outputs follow query-then-fill: pass NULL (or cap = 0) to learn the required size.
 *   - Objects returned through an out-parameter (pasur_ctx, pasur_tree) are owned by the caller
 *     and released with pasur_destroy / pasur_tree_free.  A tree must be freed before its ctx.
 *   - Cards are ids 0..51, id = 4*rank + suit, rank 0 = Ace .. 9 = Ten, 10 = Jack, 11 = Queen,
 *     12 = King; suit 0 = clubs, 1 = diamonds, 2 = hearts, 3 = spades (the paper's Fig.
 *     "Mapping Cards to Indices").  A card set is a uint64_t with bit id set.
 *   - Player 0 (Alex) moves first in every round; utilities are Alex's points minus Bob's.
 */
#ifndef PASUR_H
#define PASUR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pasur_ctx pasur_ctx;   /* one device + one stream + a device-memory budget */
typedef struct pasur_tree pasur_tree; /* one round: game tree, full game tree, CFR state  */

typedef enum {
    PASUR_OK = 0,
    PASUR_EINVAL = -1,    /* bad argument (sizes, round index, unsorted roots, wrong phase)  */
    PASUR_ENOMEM = -2,    /* device allocation failed or would exceed the ctx budget          */
    PASUR_EOVERFLOW = -3, /* a size does not fit its index type or a caller buffer (cap)      */
    PASUR_ECUDA = -4,     /* a CUDA runtime call failed; the message names it                 */
    PASUR_ETIMEOUT = -5,  /* a bounded device wait gave up                                     */
    PASUR_ENUMERIC = -6,  /* a non-finite value appeared in the CFR sweep                      */
    PASUR_ENOTIMPL = -7
} pasur_status;

/* Score inherited from earlier rounds: one row of the paper's score tensor t_scr (Table
 * "Column definitions for the score tensor"): Alex clubs, Bob clubs, point difference
 * (Alex minus Bob), 7-clubs bonus (0 none, 1 Alex, 2 Bob).  Normalised: once a bonus is
 * recorded both club counts are 0 (section "Score Tensors"). */
typedef struct {
    int16_t a_clubs, b_clubs, delta, bonus;
} pasur_score;

/* Solver settings.
 *   variant      0 = vanilla CFR (eq. RM + eq. avsigma), 1 = DCFR (eqs. DFCR_REG / DFCR_AVG)
 *   iters        number of iterations run by one pasur_cfr_iterate call (>= 0)
 *   rm_deadzone  tau: a cumulative regret counts as positive only above tau * t * Umax,
 *                Umax = max |leaf value| in the subtree of the FGT root being solved (so each
 *                root's solve depends on its own subtree only), t = iteration index (1-based)
 *   dcfr_alpha/beta/gamma  DCFR discount exponents (the paper ran 1.5, 0, 2)
 *   slots_per_item  score slots solved together by one thread block: 0 = automatic (the
 *                smallest shared-memory class a root fits with one slot, then as many slots as
 *                that class holds, at most 32); n > 0 = up to n (at most the root's own and 32),
 *                in the smallest class that holds them.  Every block takes a power-of-two number
 *                of slots; results do not depend on the grouping
 *   threads      threads per block of the CFR kernel (0 = choose per subtree size, else a
 *                multiple of 32 up to 1024)
 *   split_bytes  a root subtree whose state needs more shared memory than one block has is split
 *                over a thread-block cluster (up to 16 SMs, distributed shared memory); with
 *                split_bytes > 0 every subtree needing more than that many bytes is split too
 *                (0 = only those that do not fit).  Results do not depend on the split.
 *   stream_bytes a root subtree that does not fit one block's shared memory and has at least 16
 *                score slots, or fits no cluster either, is solved by a level-streaming sweep over
 *                every SM (state in device memory, one launch per level step); with
 *                stream_bytes > 0 every subtree needing more than that many bytes is streamed
 *                (0 = the default rule).  Results do not depend on the path.
 *   merge_delta  1 (default): the score slots of a root that differ only in the inherited point
 *                difference are solved once and share their results (average strategies, root
 *                utilities): no utility contains the inherited difference (eq. final_util,
 *                eq. passuputil), so their leaf values and hence their CFR runs coincide bit for
 *                bit.  A non-final round merges only when the next-round utilities it is given
 *                agree between such slots (checked on the first pasur_cfr_iterate call); 0 = solve
 *                every slot.  Results do not depend on it.
 */
typedef struct {
    int32_t variant;
    int32_t iters;
    float rm_deadzone;
    float dcfr_alpha, dcfr_beta, dcfr_gamma;
    int32_t slots_per_item;
    int32_t threads;
    int32_t split_bytes;
    int32_t stream_bytes;
    int32_t merge_delta;
} pasur_config;

/* Fill *cfg with the defaults: vanilla, 1000 iterations, tau = 1e-6, DCFR (1.5, 0, 2), slots that
 * differ only in delta merged. */
int pasur_config_default(pasur_config *cfg);

/* Create a context on CUDA device `device`.  hbm_budget_bytes = 0 means no limit beyond the
 * device's memory.  cuda_stream is a cudaStream_t (NULL = a new non-blocking stream owned by
 * the context).  The context's device memory comes from its own stream-ordered pool: memory a
 * freed tree or batch held stays reserved for the context's next allocations (no new mappings
 * per solve) and returns to the device at pasur_destroy; the budget counts live allocations. */
int pasur_create(pasur_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream);
/* Release the context.  EINVAL (and nothing is released) while trees of the context are alive. */
int pasur_destroy(pasur_ctx *ctx);

/* Message of the last failed call on ctx (or of the last failed pasur_create when ctx is NULL).
 * The string is owned by the library and valid until the next call on ctx. */
const char *pasur_last_error(const pasur_ctx *ctx);

/* Bytes of device memory the context holds now and at its peak. */
int pasur_memory(const pasur_ctx *ctx, size_t *in_use, size_t *peak);

/* Number of CUDA kernels launched through ctx since its creation (host out). */
int pasur_launch_count(const pasur_ctx *ctx, int64_t *count);

/* Seeded deal (section "Pasur", initial pool rule): SplitMix64-seeded xoshiro256**,
 * unbiased Fisher-Yates over 0..51 (i = 51..1, j uniform in [0, i]); deck[0:4] is the initial
 * pool and holds no Jack: one Jack is swapped with deck[4] unless deck[4] is a Jack too, and two
 * or more Jacks force a fresh shuffle of 0..51 with the stream continued.  Round r (0..5) deals
 * deck[4+8r : 8+8r] to Alex and deck[8+8r : 12+8r] to Bob.  Host only; deck_out is host memory. */
int pasur_deal(uint64_t seed, uint8_t deck_out[52]);

/* Build the level-ordered game tree (GT) of round `round` (0..5; 5 = final) for the given root
 * pools (section "Actions", CodeSnippet "ApplyActions", Table "Capture rules for each card type").
 * root_pools (host or device): n_pools card sets, strictly ascending, disjoint from the round's
 * hands.  Level 0 holds the roots; level k+1 holds the children of level k's nodes in parent
 * order, each node's children sorted by (played card, picked set as an integer).  Legal moves:
 * a numeric card takes any nonempty set of pool numerics completing its value to 11 (one move per
 * set) or, with none, is laid; a Jack takes every pool card that is not a King or Queen (laid if
 * there is none); a Queen or King takes one pool card of its rank (one move each) or is laid.
 * Errors: EINVAL (round, unsorted/overlapping pools), ENOMEM, EOVERFLOW. */
int pasur_build_round(pasur_ctx *ctx, const uint8_t deck[52], int round, const uint64_t *root_pools,
                      int64_t n_pools, pasur_tree **out);
int pasur_tree_free(pasur_tree *tree);

/* GT level sizes and, once unfolded, full-game-tree (FGT) level sizes (-1 before).  Host out. */
int pasur_tree_sizes(const pasur_tree *tree, int64_t gt_sizes[9], int64_t fgt_sizes[9]);

/* Unfolding Process (section "In-Hand Updates", Fig. "Unfolding Process"): GT root g carries the
 * score slots score_offs[g] .. score_offs[g+1]-1 of `scores`; every FGT level lists, for each GT
 * node of the level in order, one node per slot of its root (GT-major, slot-minor), so FGT node
 * (j, s) has parent (parent(j), s).  score_offs: n_pools+1 int64 (host), scores: host array.
 * Scores of one root must be strictly ascending in (a_clubs, b_clubs, delta, bonus) order.
 * level_sizes_out (host, may be NULL) receives the 9 FGT level sizes.  Resets any CFR state. */
int pasur_unfold(pasur_tree *tree, const int64_t *score_offs, const pasur_score *scores,
                 int64_t level_sizes_out[9]);

/* Run cfg->iters iterations of CFR on an unfolded round (section "CFR Algorithm"): each FGT node
 * is its own information set; root reach 1 for both players; per iteration regret matching
 * (eq. RM, with the cfg dead zone), reach top-down, values bottom-up, then R(h,a) +=
 * s_p pi_{-p}(h) (v(h.a) - v(h)) and S(h,a) += pi_p(h) sigma(h,a) (eq. avsigma) for every edge,
 * and the root value is accumulated.  The first call after pasur_unfold fixes the leaf values:
 * final round: this round's point difference after CleanUp plus +7 / -7 for the 7-clubs bonus
 * (eq. final_util); other rounds: the round's point difference plus next_root_util[lnk(leaf)]
 * (eq. passuputil), with the links of pasur_next_roots (which must have been called).
 * next_root_util: float per next-round FGT root, host or device; NULL for the final round; it is
 * read only on the first call.  Later calls continue the same run.  Errors: EINVAL, ENUMERIC. */
int pasur_cfr_iterate(pasur_tree *tree, const pasur_config *cfg, const float *next_root_util);

/* pasur_cfr_iterate on the GT roots root_first .. root_first + root_count - 1 only: the roots of a
 * round are independent (open hands, root reach 1), so several solvers can each take a range and
 * add their root utilities (every root outside a solver's range has utility 0 there, so the sum of
 * the solvers' pasur_round_utilities outputs is the whole round's, bit for bit).  Average
 * strategies outside the range are unspecified.  The range is fixed by the first call on the tree
 * (EINVAL if a later call passes another); pasur_cfr_iterate continues with it. */
int pasur_cfr_iterate_roots(pasur_tree *tree, const pasur_config *cfg, const float *next_root_util,
                            int64_t root_first, int64_t root_count);

/* Number of GT nodes (all levels) below every GT root (host out, cap >= GT roots): the size by
 * which callers balance root ranges. */
int pasur_root_sizes(const pasur_tree *tree, int64_t *gt_nodes_out, int64_t cap);

/* Average strategy (eq. avsigma, normalised per FGT parent; uniform where the strategy sum is 0)
 * of every FGT edge: levels 1..8 concatenated, each level in FGT order.  out: float, host or
 * device, cap = its length in elements (>= sum of FGT level sizes 1..8, else EOVERFLOW). */
int pasur_avg_strategy(const pasur_tree *tree, float *out, int64_t cap);

/* Average root utility of every FGT root (sum over iterations of v(root), divided by the number
 * of iterations; CodeSnippet "CFR").  out: float, host or device, cap >= FGT level-0 size. */
int pasur_round_utilities(const pasur_tree *tree, float *out, int64_t cap);

/* pasur_avg_strategy without waiting: the strategies are computed on the context's stream and,
 * for host memory, copied to out on a copy stream of the context that runs beside the context's
 * later work (the next round's CFR); for device memory the call is ordered on the context's
 * stream.  out must stay valid and unread until pasur_sync(ctx) returns; a host buffer should be
 * page-locked for the copy to overlap.  Same layout and errors as pasur_avg_strategy. */
int pasur_avg_strategy_async(const pasur_tree *tree, float *out, int64_t cap);

/* Wait for everything the context queued: its stream and the copies of asynchronous exports. */
int pasur_sync(pasur_ctx *ctx);

/* Between-hand update (section "Between-Hand Updates", CodeSnippet "BetweenHands"): the next
 * round's FGT roots.  For every FGT leaf (j, s) the next root is (pool at j, normalise(score s +
 * the round's clubs and point difference at j)).  Roots: unique pools ascending, per pool unique
 * scores ascending.  Outputs (host; any may be NULL to query): pools_out[n_pools],
 * score_offs_out[n_pools+1], scores_out[n_roots], lnk_out[FGT leaves] (index of each leaf's next
 * root, the paper's t_lnk).  The links are also kept on the device for pasur_cfr_iterate.
 * cap_pools / cap_roots bound the two arrays; too small -> EOVERFLOW with the sizes still set.
 * Not valid for the final round (EINVAL). */
int pasur_next_roots(pasur_tree *tree, uint64_t *pools_out, int64_t cap_pools, int64_t *score_offs_out,
                     pasur_score *scores_out, int64_t cap_roots, int64_t *lnk_out, int64_t *n_pools,
                     int64_t *n_roots);

/* Export GT level k (0..8) for parity checks; every output is host memory and may be NULL:
 * parent[n] (int64, level k-1 index; -1 at level 0), nchild[n] (int32; 0 at level 8),
 * lay[n] (int32 card played into the node; -1 at level 0), pick[n] (uint64 picked set),
 * state[3n] (Alex hand, Bob hand, pool), rus[7n] (int8 running score: Alex clubs, Bob clubs,
 * last picker 0/1/2, Alex points, Alex surs, Bob points, Bob surs).  cap = n of the caller. */
int pasur_export_level(const pasur_tree *tree, int k, int64_t cap, int64_t *parent, int32_t *nchild,
                       int32_t *lay, uint64_t *pick, uint64_t *state, int8_t *rus);

/* Export the FGT leaf values fixed by the first pasur_cfr_iterate call (float per FGT leaf,
 * host or device).  EINVAL before that call. */
int pasur_leaf_values(const pasur_tree *tree, float *out, int64_t cap);

/* Convergence of the average strategy (section "Experimental Evaluation", figure "Convergence of
 * CFR": the mean squared error of each intermediate average strategy to the final one, per round).
 * Continues the CFR run of the tree (as pasur_cfr_iterate with cfg, cfg->iters ignored) up to each
 * of the n iteration counts checkpoints[0] < ... < checkpoints[n-1] (counted from the start of the
 * run; the first must exceed the iterations already done) and keeps the average strategy there.
 * mse_out[i] (host, n doubles) = mean over every FGT edge (levels 1..8) of
 * (sigma-bar after checkpoints[i] - sigma-bar after checkpoints[n-1])^2, so mse_out[n-1] = 0.
 * next_root_util as in pasur_cfr_iterate.  Holds n copies of the average strategy of the solved
 * slots on the device during the call.  Errors: EINVAL (checkpoints), ENOMEM, ENUMERIC. */
int pasur_cfr_convergence(pasur_tree *tree, const pasur_config *cfg, const float *next_root_util,
                          const int64_t *checkpoints, int n, double *mse_out);

/* Work the CFR solve of a tree does (after its first pasur_cfr_iterate): solved_sizes (host, may be
 * NULL) receives the 9 FGT level sizes over the solved slots (cfg.merge_delta; equal to the FGT
 * sizes without merging), swept_edges (may be NULL) the (node, solved slot) pairs below the roots
 * that carry CFR state: the children of nodes with more than one path below them.  Every other
 * edge lies on a forced-move chain (average strategy 1, regret 0, never touched per iteration). */
int pasur_solved_sizes(const pasur_tree *tree, int64_t solved_sizes[9], int64_t *swept_edges);

/* Checkpoint and resume of a round's CFR (the paper keeps each round's state in host memory and
 * stores solved profiles, section "Experimental Evaluation").  After the tree's CFR has been set
 * up (its first pasur_cfr_iterate; iters 0 allowed), pasur_save_round writes the round's regrets,
 * strategy sums, root-value sums, iteration count and variant, after a header of sizes and a hash
 * of its leaf values, into buf (host memory, cap bytes); with buf NULL it only sets *bytes to the
 * size it needs.  pasur_load_round restores such a checkpoint into a tree built, unfolded and set
 * up the same way (same deal, round, roots, score slots, next-round utilities, variant and solver
 * settings): the next pasur_cfr_iterate continues the saved run as if it had not stopped, bit for
 * bit.  buf: host memory, read or written only during the call.  Errors: EINVAL (no CFR set-up,
 * cap too small, not a checkpoint, truncated, or a header or leaf hash that differs from the
 * tree's), ECUDA. */
int pasur_save_round(const pasur_tree *tree, void *buf, size_t cap, size_t *bytes);
int pasur_load_round(pasur_tree *tree, const void *buf, size_t bytes);

/* The (active node, solved slot) pairs the CFR updates per iteration (after the first
 * pasur_cfr_iterate; host out): one regret-matching step in the top-down pass and one value, regret
 * and strategy-sum update in the bottom-up pass each.  With pasur_solved_sizes' swept edges this is
 * the kernel's work per iteration (its shared-memory traffic is about 28 B per swept edge plus 32 B
 * per pair).  EINVAL: NULL out, no CFR run yet. */
int pasur_swept_pairs(const pasur_tree *tree, int64_t *swept_pairs);

/* How the CFR solves each GT root (after the first pasur_cfr_iterate; host out, cap >= GT roots):
 * 0..4 = one thread block per item with the state in shared memory (size classes, smallest
 * first), 5 = the level-streaming sweep over every SM with the state in device memory, 6 = a
 * thread-block cluster (the subtree split over several SMs' shared memory), -1 = no CFR work
 * (no score slot, or no move).  A diagnostic: results do not depend on the path. */
int pasur_root_paths(const pasur_tree *tree, int32_t *path_out, int64_t cap);

/* Timing of the last pasur_cfr_iterate call on the device (CUDA events around the CFR kernel
 * launches), the number of FGT edges, and the kernel launches it made. */
int pasur_last_cfr_stats(const pasur_tree *tree, float *ms, int64_t *edges, int32_t *launches);

/* ---- batched exact solve of many deals ---------------------------------------------------- */
typedef struct pasur_batch pasur_batch;

/* Build rounds first_round..5 of n_deals seeded deals (decks: host, 52 bytes per deal), each from
 * the standalone root of first_round (pool = deck[0:4], score (0,0,0,0)), with every round's
 * unfolding and links, and plan their CFR: the work items of all deals' trees of one round are
 * merged into one persistent launch per shared-memory class (largest subtrees first).  With
 * cfg->threads == 0 an autotuner times candidate block sizes per class on the round with the most
 * work and keeps the fastest.  cfg is fixed for the batch.  The batch owns its trees.
 * The deals are built on up to 8 host threads (at most one per deal and per host core; the
 * environment variable PASUR_BUILD_WORKERS lowers the count), each on its own CUDA stream; the
 * result does not depend on the count.  Their device memory counts against ctx's budget; on any
 * error (the first failing deal's message in pasur_last_error) nothing of the batch is left. */
int pasur_batch_create(pasur_ctx *ctx, const uint8_t *decks, int64_t n_deals, int first_round, const pasur_config *cfg,
                       pasur_batch **out);

/* The surrogate-plus-batched form: rounds first_round..last_round only; the leaves of last_round
 * (< 5) take their next-round values from the surrogate's predictions for the roots that follow
 * (pasur_mlp_predict_next, computed here once), so the later rounds are never built.  With
 * last_round = 5, mlp may be NULL and this is pasur_batch_create.  pasur_batch_selfplay needs
 * last_round = 5.  (pasur_mlp is declared below.) */
struct pasur_mlp;
int pasur_batch_create_cut(pasur_ctx *ctx, const uint8_t *decks, int64_t n_deals, int first_round, int last_round,
                           const pasur_config *cfg, struct pasur_mlp *mlp, pasur_batch **out);

/* pasur_batch_create with given roots: deal d's round first_round starts from the pools
 * pools[deal_roots[d] .. deal_roots[d+1]) (strictly ascending per deal), pool i carrying the score
 * slots scores[score_offs[i] .. score_offs[i+1]) (ascending, as for pasur_unfold); rounds
 * first_round..5 are built and solved as in pasur_batch_create.  Roots are independent, so each
 * root's utility equals its utility in a batch over all roots.  All arrays host;
 * deal_roots: n_deals + 1 entries, score_offs: deal_roots[n_deals] + 1 entries. */
int pasur_batch_create_roots(pasur_ctx *ctx, const uint8_t *decks, int64_t n_deals, int first_round, const int64_t *deal_roots,
                             const uint64_t *pools, const int64_t *score_offs, const pasur_score *scores,
                             const pasur_config *cfg, pasur_batch **out);

/* Replace the values the leaves of a cut batch's last round take at the roots after the cut
 * (pasur_batch_create_cut: the surrogate's predictions): values (host or device, n floats, n =
 * the number of roots pasur_next_roots gives for that deal's last tree) for deal `deal`.  The
 * next pasur_batch_solve uses them (the solve graph reads the same buffer). */
int pasur_batch_set_cut_values(pasur_batch *b, int64_t deal, const float *values, int64_t n);

/* Solve the batch from scratch: cfg->iters CFR iterations per round, round 5 first, each round's
 * leaf values from the next round's average root utilities (eq. passuputil).  The first call
 * captures the whole backward sweep into a CUDA graph; every call replays it.  root_util_out
 * (host or device, may be NULL): the average utility of every deal's root of first_round. */
int pasur_batch_solve(pasur_batch *b, float *root_util_out, int64_t cap);

/* Borrow the tree of (deal, round) for pasur_avg_strategy, pasur_round_utilities, pasur_tree_sizes
 * and the exports; it stays owned by the batch (do not free it). */
int pasur_batch_tree(const pasur_batch *b, int64_t deal, int round, pasur_tree **tree_out);

/* Device time of the last pasur_batch_solve (CUDA events around the graph launch), the number of
 * FGT edges of all trees, and the kernel launches in one solve. */
int pasur_batch_stats(const pasur_batch *b, float *ms, int64_t *edges, int64_t *launches);
/* The work of one pasur_batch_solve, summed over all trees as in pasur_solved_sizes: FGT edges over
 * the solved slots, and the swept (node, solved slot) pairs that carry CFR state. */
int pasur_batch_work(const pasur_batch *b, int64_t *solved_edges, int64_t *swept_edges);
/* The (active node, solved slot) pairs of one pasur_batch_solve iteration, summed over all trees
 * as in pasur_swept_pairs.  EINVAL: NULL batch or out. */
int pasur_batch_pairs(const pasur_batch *b, int64_t *swept_pairs);
int pasur_batch_free(pasur_batch *b);

/* ---- self-play (fair value) ---------------------------------------------------------------- */
/* Sampled games: the paper estimates the fair value of a deal by playing many games on the GPU
 * between strategy profiles (§Introduction, learned-strategy study), every move drawn at the node
 * reached, one choice per parent (§External Sampling).
 *
 * pasur_selfplay plays n_games games from FGT root root_q of rounds[0] through the n_rounds trees
 * rounds[0..n_rounds) (host array): consecutive rounds of one deal, the last one round 5, each
 * non-final tree with pasur_next_roots called and the next tree unfolded over exactly the roots
 * it returned (EINVAL when the sizes disagree).  sigma: NULL or a host array of n_rounds
 * pointers; entry i NULL uses tree i's average strategy (its CFR run), else the strategy of every
 * FGT edge of round i in the pasur_avg_strategy layout (float, host or device, read only during
 * the call).  Move rule, in float arithmetic, at ply p of game g (plies numbered from 0 across the
 * rounds): u = the top 24 bits of word 0 of Philox4x64-10 (Salmon et al., SC 2011) at counter
 * (p, g, 0, 0) under key (seed, 0), times 2^-24; w_a = the strategies of the node's children in
 * canonical order; total = w_0 + w_1 + ... (left to right); the move is the first a with
 * w_0 + ... + w_a > u * total; if there is none, the last a with w_a > 0, else a = 0.
 * out: int16 per game (host or device): the final game difference, Alex minus Bob points of the
 * whole game including root_q's inherited difference and the 7-clubs bonus.  Game g depends only
 * on (seed, g), not on n_games.  Errors: EINVAL (arguments above, missing CFR run), ENOMEM. */
int pasur_selfplay(pasur_ctx *ctx, pasur_tree *const *rounds, int n_rounds, const float *const *sigma, int64_t root_q,
                   int64_t n_games, uint64_t seed, int16_t *out);

/* The same over a solved batch: n_games games per deal from its first round's root with the
 * batch's average strategies, deal d under seeds[d] (host, n_deals), all deals in one launch.
 * out: int16 [n_deals * n_games] deal-major, host or device.  EINVAL before pasur_batch_solve. */
int pasur_batch_selfplay(pasur_batch *b, int64_t n_games, const uint64_t *seeds, int16_t *out);

/* Device time (CUDA events around the self-play kernel) and number of games of the context's last
 * pasur_selfplay or pasur_batch_selfplay call. */
int pasur_last_selfplay_stats(const pasur_ctx *ctx, float *ms, int64_t *games);

/* ---- game values under fixed or optimal play (exploitability) ---------------------------- */
/* Probability of reaching every next-round FGT root when both players follow sigma (NULL = the
 * tree's own average strategy; else host or device, the pasur_avg_strategy layout) from the
 * round's FGT roots with reach root_reach (double per FGT root, host or device; NULL = 1 each):
 * the reach of every FGT leaf summed into its next root (t_lnk).  Chained over rounds it gives the
 * probability of every later round's root under a strategy profile.  next_reach: double [next
 * roots], host or device.  Non-final rounds after pasur_next_roots only. */
int pasur_round_reach(pasur_tree *tree, const float *sigma, const double *root_reach, double *next_reach, int64_t cap);

/* fp64 value of every FGT root of a round, from its leaves up: mode 0 minimax (Alex maximises,
 * Bob minimises), 1 Alex's best response to Bob's strategy, 2 Bob's best response to Alex's, 3 both
 * following the strategy.  Leaves as in pasur_cfr_iterate: final round = the round's difference
 * after CleanUp + bonus; other rounds = the round's difference + next_values[lnk(leaf)]
 * (next_values: double per next-round FGT root, host or device; NULL for the final round).
 * sigma: strategy of every FGT edge in the pasur_avg_strategy layout (host or device), or NULL to
 * use the tree's own average strategy; unused in mode 0.  Chaining mode 1 (resp. 2) from round 5
 * down to round 0 gives the best-response values BR_A >= v >= BR_B of a whole-game profile; its
 * exploitability is (BR_A - BR_B) / 2.  Expected values are summed child by child in canonical
 * order (no fused multiply-add).  out: double [FGT roots], host or device. */
int pasur_root_values(pasur_tree *tree, int mode, const float *sigma, const double *next_values, double *out, int64_t cap);

/* Probability of every next-round root when one player best-responds and the other follows sigma:
 * mode 1 Alex best-responds, 2 Bob does, 3 both follow sigma (as pasur_round_reach).  The
 * responder's move at each of its nodes is the choice of the value pass of pasur_root_values with
 * the same mode, sigma and next_values (the first best child in canonical order); reach is
 * multiplied in fp64.  root_reach: double per FGT root of this round, host or device (NULL = 1
 * each); next_values: double per next-round FGT root, host or device (required); next_reach:
 * double [next roots], host or device.  Non-final rounds after pasur_next_roots only. */
int pasur_response_reach(pasur_tree *tree, int mode, const float *sigma, const double *next_values,
                         const double *root_reach, double *next_reach, int64_t cap);

/* ---- round-start utility surrogate ---------------------------------------------------------- */
/* A 256-256-256-256-1 network (GELU hidden layers) that predicts the average utility U of a
 * round-start FGT root, so that a round's leaves can take their next-round values (eq.
 * passuputil) without the later rounds being built and solved.  The paper's learned part is a
 * gradient-boosted model of the strategy (§Results); this surrogate is trained on the U values
 * the exact solver produces; the exact solve is its fallback and measures its error.  Weights are stored in
 * f32 (Adam state in f32) and used as bf16 by the tensor-core kernels, which accumulate in f32.
 *
 * Input features of a root of round r with pool P and score (ac, bc, delta, bonus), 256 values,
 * exactly representable in bf16: [52*loc + card] = 1 for every card, loc 0 = Alex (in Alex's
 * hands of rounds r..5, i.e. deck[4+8i .. 8+8i] for i >= r), 1 = Bob (deck[8+8i .. 12+8i]),
 * 2 = in P, 3 = out (captured before round r); [208] = ac/8, [209] = bc/8, [210] = delta/32,
 * [211 + bonus] = 1, [214 + r] = 1; for loc = 0, 1, 2: [220 + 4 loc] = clubs / 8, [221 + 4 loc] =
 * points / 8 (Aces and Jacks 1, two of clubs 2, ten of diamonds 3), [222 + 4 loc] = Jacks / 4,
 * [223 + 4 loc] = cards / 32 of that location; [232..255] = 0.
 * Flat parameter layout (f32, 197,377 values): W0 [256 x 256] (row = output unit), b0 [256],
 * W1, b1, W2, b2, w3 [256], b3 [1]; y = w3 . h3 + b3, h(l+1) = gelu(W_l h_l + b_l), h0 = x,
 * gelu(z) = z * Phi(z). */
typedef struct pasur_mlp pasur_mlp;

/* dataset_capacity: rows of the on-device training set (features bf16 + targets f32).  Weights
 * are drawn Uniform(-1/16, 1/16) from SplitMix64(seed), biases 0. */
int pasur_mlp_create(pasur_ctx *ctx, int64_t dataset_capacity, uint64_t seed, pasur_mlp **out);
int pasur_mlp_free(pasur_mlp *mlp);
/* Replace / read all parameters (flat layout above; host or device).  Setting resets Adam. */
int pasur_mlp_set_params(pasur_mlp *mlp, const float *params, int64_t n);
int pasur_mlp_get_params(const pasur_mlp *mlp, float *params, int64_t cap);
/* Predictions for n feature rows (x: bf16 bit patterns, row-major [n x 256], host or device;
 * y_out: float [n], host or device). */
int pasur_mlp_forward(pasur_mlp *mlp, const uint16_t *x, int64_t n, float *y_out);
/* Mean squared error over n <= 2^20 rows against targets y and its gradient with respect to every
 * parameter (flat layout), without updating anything; loss_out / grads_out may be NULL. */
int pasur_mlp_gradients(pasur_mlp *mlp, const uint16_t *x, const float *y, int64_t n, float *loss_out, float *grads_out);
/* Append every FGT root of a solved tree (features of its pools and score slots, target = its
 * average utility) to the training set.  EOVERFLOW beyond the capacity. */
int pasur_mlp_dataset_add_tree(pasur_mlp *mlp, const pasur_tree *tree);
/* Append n rows given directly (x: bf16 bit patterns [n x 256], y: float [n]; host or device). */
int pasur_mlp_dataset_add_rows(pasur_mlp *mlp, const uint16_t *x, const float *y, int64_t n);
int pasur_mlp_dataset_size(const pasur_mlp *mlp, int64_t *n);
int pasur_mlp_dataset_export(const pasur_mlp *mlp, int64_t first, int64_t count, uint16_t *x_out, float *y_out);
int pasur_mlp_dataset_clear(pasur_mlp *mlp);
/* Adam (lr, beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared error over the training set:
 * `epochs` passes, each over a fresh shuffle (SplitMix64(shuffle_seed) Fisher-Yates) in batches
 * of `batch` rows (a multiple of 128, <= 65536; the last batch may be partial).  One CUDA graph
 * per epoch.  epoch_loss_out (host, may be NULL): mean batch loss of every epoch. */
int pasur_mlp_train(pasur_mlp *mlp, int epochs, int64_t batch, float lr, uint64_t shuffle_seed, float *epoch_loss_out);
/* Predicted U of every next-round FGT root of a non-final tree (after pasur_next_roots), in the
 * order of pasur_next_roots: pass the result to pasur_cfr_iterate as next_root_util. */
int pasur_mlp_predict_next(pasur_mlp *mlp, const pasur_tree *tree, float *out, int64_t cap);
/* Features of arbitrary roots of round `round` of a deal (pools[n_pools], score_offs[n_pools+1],
 * scores; host) as bf16 rows [score_offs[n_pools] x 256] into x_out (host or device). */
int pasur_mlp_root_features(pasur_ctx *ctx, const uint8_t deck[52], int round, const uint64_t *pools,
                            const int64_t *score_offs, const pasur_score *scores, int64_t n_pools, uint16_t *x_out);
/* Device time of the last pasur_mlp_train call and the Adam steps taken so far. */
int pasur_mlp_stats(const pasur_mlp *mlp, float *last_train_ms, int64_t *adam_steps);

/* Exclusive prefix sum of per-node move counts into CSR child offsets, allocating nothing.
 * This is the step between the count and emit passes of the level expansion; the paper has no
 * counterpart (its expansion runs on PyTorch tensor ops).  It exists for callers that cannot
 * allocate device memory at the point of the call: applications that give all GPU memory to their
 * own arena, plug-ins inside a host program that owns the allocator, code that must not risk an
 * out-of-memory failure or the allocator's locks mid-run.  pasur_build_round does the same step
 * with scratch it allocates; this variant uses a fixed 32 KB array compiled into the library
 * (every GPU that loads the library holds it until the process exits).
 *   counts   device, n int32 (each >= 0); offsets: device, n+1 int64, offsets[i] = sum of
 *            counts[0..i), offsets[n] = total.  Both stay owned by the caller.
 *   n        0 <= n <= 4,194,303, else PASUR_EOVERFLOW (pasur_last_error(NULL) says why).
 *            counts and offsets must be device (or managed) memory, else PASUR_EINVAL; the
 *            length of offsets cannot be checked here: it must hold n+1 elements.
 *   cuda_stream  cudaStream_t the work is queued on (NULL = the legacy default stream); the call
 *            returns without waiting.  Queue it after the work that writes counts.
 * The first call made in a CUDA context (normally: the first call with a given device current)
 * looks up the array's device address (cudaGetSymbolAddress) and caches it for that context;
 * make that first call outside any stream capture.  All calls share the array: two calls that
 * overlap on the GPU (other streams, or other host threads on the same stream without ordering)
 * race and may return wrong offsets. */
int pasur_move_offsets_noalloc(const int32_t *counts, int64_t n, int64_t *offsets, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* PASUR_H */
