/*
 * wcc_oracle.h -- plain CPU oracle for Well-Connected Clusters refinement.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA path, and the CUDA path never
 * calls it.
 *
 * What it computes (paper: Section 2.2 Algorithm 1 "CCR", Section 2.3
 * Algorithms 2-3 "WCC" / "isWCC", criterion f(n) of Section 2 with log10 n as
 * used in Section 3; Section 2.4 Algorithms 4-5 "CM" with a CPM community
 * step), under these readings where the paper is silent:
 *   - threshold: a cluster of n vertices fails iff its min cut <= T(n), with
 *     T(n) the exact integer form of the criterion (floor(log10 n) for LOG10);
 *   - peeling: round-synchronous removal of every vertex whose degree inside
 *     the cluster is <= T(|S|), T recomputed each round, to a fixpoint;
 *   - min cut: Nagamochi-Ibaraki contraction with k = T+1 (maximum-adjacency
 *     orderings, keys capped at k, ties to the smallest id) to a fixpoint,
 *     then canonical Stoer-Wagner on the contracted graph (ties to the
 *     smallest super-vertex id, earliest phase attaining the minimum kept,
 *     the side is the last-added super-vertex, never the one holding local 0);
 *   - sizes: a part is kept iff |part| >= min_size  (s_pre = s_post = min_size-1);
 *   - output ids: accepted clusters numbered 0..K-1 in ascending order of
 *     their smallest vertex id, -1 for every other vertex.
 * All arithmetic is integer.
 */
#ifndef WCC_ORACLE_H
#define WCC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { WO_RULE_LOG10 = 0, WO_RULE_LOG2 = 1, WO_RULE_SQRT = 2, WO_RULE_LINEAR = 3 };

typedef struct {
  int64_t in_clusters;     /* distinct input labels >= 0 holding at least one vertex */
  int64_t out_clusters;    /* accepted clusters */
  int64_t items;           /* work items processed (after CCR) */
  int64_t splits;          /* items whose min cut was <= T and were bisected */
  int64_t peeled;          /* vertices removed by peeling */
  int64_t ni_passes;       /* maximum-adjacency passes of the contraction */
  int64_t sw_phases;       /* Stoer-Wagner phases */
} wo_stats;

/* Largest integer T with "cut <= T  <=>  cut <= f(n)" for integer cuts.
 * LOG10: floor(log10 n); LOG2: floor(log2 n); SQRT: floor(sqrt n);
 * LINEAR: floor(num*n/den).  n < 1 gives -1 (no degree is <= -1). */
int64_t wo_threshold(int32_t kind, int64_t num, int64_t den, int64_t n);

/* Simple undirected CSR from an edge list: both directions, self-loops and
 * duplicates dropped, rows sorted.  off has n+1 entries, adj room for 2m.
 * Returns 0, or -1 on an id outside [0,n). */
int wo_build_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                 int64_t *off, int32_t *adj, int64_t *nnz);

/* Connected components of a graph given as an edge list on ids 0..n-1:
 * comp[v] = smallest vertex id in v's component.  Returns the count. */
int64_t wo_components(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                      int32_t *comp);

/* Round-synchronous peel of a whole graph (edge list, ids 0..n-1) under the
 * rule.  alive[v] = 1 for survivors.  Returns the number of survivors. */
int64_t wo_peel(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                int32_t kind, int64_t num, int64_t den, uint8_t *alive);

/* Canonical Stoer-Wagner on a connected weighted graph (edge list, ids
 * 0..n-1, w may be NULL for unit weights, n >= 2).  side[v] = 1 on the
 * returned side.  Returns the min cut value, or -1 if n < 2. */
int64_t wo_stoer_wagner(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                        const int64_t *w, uint8_t *side);

/* The cut step of one work item on a connected simple graph (edge list, ids
 * 0..n-1, n >= 2) with threshold T: contraction with k = T+1 to a fixpoint,
 * then, if more than one super-vertex remains, canonical Stoer-Wagner on the
 * contracted graph.  rep[v] = super-vertex (smallest id) of v after the
 * contraction.  Returns 1 (accept: min cut > T) or 0 (fail: *lambda = min
 * cut, side[v] = 1 on the cut side).  Returns -1 on bad input. */
int wo_item_cut(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev, int64_t T,
                int32_t *rep, uint8_t *side, int64_t *lambda);

/* Full WCC refinement (Algorithm 2 with CCR first, then per item: peel, CC,
 * cut).  label_in[v] >= 0 is v's input cluster, -1 none.  Only input labels
 * with only_label[label] != 0 are refined when only_label is non-NULL and
 * label values are < n_only (used for sampled checks of large inputs).
 * out_mode 0: label_out = accepted-cluster rank by smallest vertex id;
 * out_mode 1: label_out = smallest vertex id of the accepted cluster.
 * Returns 0, or -1 on bad input. */
int wo_wcc(int64_t n, const int64_t *off, const int32_t *adj, const int32_t *label_in,
           int32_t kind, int64_t num, int64_t den, int32_t min_size,
           const uint8_t *only_label, int64_t n_only, int32_t out_mode,
           int32_t *label_out, wo_stats *stats);

/* The community step of CM (GetCommunities of Algorithm 5) as used here: CPM
 * local moving at resolution gamma = gnum/gden on a graph given as an edge
 * list on ids 0..n-1 (each entry counts once), in ascending-id sweeps from
 * singletons, each vertex moving to the neighbouring (or an empty) community
 * of largest gain k(v,c)*gden - gnum*n_c (ties to the smallest community id)
 * only when that beats staying, at most 64 sweeps; then, when connected is
 * nonzero (as CM uses it), every community is split into its connected
 * parts.  comm[v] = smallest id of v's community.  Returns the number of
 * communities, or -1 on bad input. */
int64_t wo_cpm_communities(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                           int64_t gnum, int64_t gden, int32_t connected, int32_t *comm);

/* CM refinement (Section 2.4, Algorithms 4-5): wo_wcc, except that each part
 * of a split with at least min_size vertices is divided into its CPM
 * communities (wo_cpm_communities on the part's induced subgraph) and every
 * community with at least min_size vertices is checked again.  Arguments as
 * wo_wcc, plus the resolution gnum/gden (gnum >= 0, gden >= 1).  Returns 0,
 * or -1 on bad input. */
int wo_cm(int64_t n, const int64_t *off, const int32_t *adj, const int32_t *label_in,
          int32_t kind, int64_t num, int64_t den, int32_t min_size, int64_t gnum, int64_t gden,
          const uint8_t *only_label, int64_t n_only, int32_t out_mode, int32_t *label_out,
          wo_stats *stats);

#ifdef __cplusplus
}
#endif
#endif
