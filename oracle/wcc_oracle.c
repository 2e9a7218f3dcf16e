/*
 * wcc_oracle.c -- plain CPU oracle for Well-Connected Clusters refinement.
 *
 * TEST INFRASTRUCTURE ONLY (see wcc_oracle.h): slow, single-threaded and
 * written to be checked against the paper by eye.  No blocking, fusion or
 * reordering beyond what the definitions below state.  Every step cites the
 * part of the paper it follows; the readings the paper leaves open are listed
 * in the header.
 */
#include "wcc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Criterion (Section 2: f(n) in {log10 n, log2 n, sqrt n, k*n}; Section 3
 * uses log10 n).  The paper accepts iff cut > f(n).  For an integer cut this
 * is cut > T(n) with T(n) the largest integer <= f(n), computed here without
 * floating point so that exact powers (n = 1000) are never misrounded. */
int64_t wo_threshold(int32_t kind, int64_t num, int64_t den, int64_t n) {
  int64_t t, p;
  if (n < 1) return -1;
  switch (kind) {
    case WO_RULE_LOG10: /* largest t with 10^t <= n */
      t = 0; p = 1;
      while (p <= n / 10) { p *= 10; t++; }
      return t;
    case WO_RULE_LOG2: /* largest t with 2^t <= n */
      t = 0; p = 1;
      while (p <= n / 2) { p *= 2; t++; }
      return t;
    case WO_RULE_SQRT: /* largest t with t*t <= n */
      t = (int64_t)sqrt((double)n);
      while (t > 0 && t * t > n) t--;
      while ((t + 1) * (t + 1) <= n) t++;
      return t;
    case WO_RULE_LINEAR: /* largest t with t*den <= num*n */
      if (den <= 0 || num < 0) return -1;
      return (num * n) / den;
    default:
      return -1;
  }
}

/* ------------------------------------------------------------------------ */
/* Graphs.  G: the whole graph as CSR on global ids.  lgraph: the subgraph of
 * one item on local ids 0..n-1 (local id = rank of the global id in the
 * item's ascending vertex list), optionally with integer edge weights. */

typedef struct {
  int64_t n;
  const int64_t *off;
  const int32_t *adj;
} graph;

typedef struct {
  int32_t n;
  int64_t *off;
  int32_t *adj;
  int64_t *wt; /* NULL: every edge has weight 1 */
} lgraph;

static void lgraph_free(lgraph *H) {
  free(H->off);
  free(H->adj);
  free(H->wt);
  H->off = NULL; H->adj = NULL; H->wt = NULL;
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

int wo_build_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                 int64_t *off, int32_t *adj, int64_t *nnz) {
  int64_t i, v, e, w;
  int64_t *fill;
  for (i = 0; i < m; i++)
    if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return -1;
  /* degree of each vertex, both directions, self-loops dropped */
  for (v = 0; v <= n; v++) off[v] = 0;
  for (i = 0; i < m; i++) {
    if (src[i] == dst[i]) continue;
    off[src[i] + 1]++;
    off[dst[i] + 1]++;
  }
  for (v = 0; v < n; v++) off[v + 1] += off[v];
  fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  for (v = 0; v <= n; v++) fill[v] = off[v];
  for (i = 0; i < m; i++) {
    if (src[i] == dst[i]) continue;
    adj[fill[src[i]]++] = dst[i];
    adj[fill[dst[i]]++] = src[i];
  }
  /* sort every row and drop repeated neighbours, compacting in place */
  w = 0;
  for (v = 0; v < n; v++) {
    int64_t b = off[v], t = off[v + 1];
    qsort(adj + b, (size_t)(t - b), sizeof(int32_t), cmp_i32);
    off[v] = w;
    for (e = b; e < t; e++)
      if (e == b || adj[e] != adj[e - 1]) adj[w++] = adj[e];
  }
  off[n] = w;
  *nnz = w;
  free(fill);
  return 0;
}

/* Induced subgraph G[S] (Algorithm 1: E_c = {(u,v) in E : u,v in V_c};
 * Algorithm 3 re-induces each side the same way).  S is ascending; pos is a
 * scratch array over all global ids holding -1 on entry and on exit. */
static void induce(const graph *G, const int32_t *S, int32_t n, int32_t *pos, lgraph *H) {
  int32_t i;
  int64_t e, cnt = 0;
  for (i = 0; i < n; i++) pos[S[i]] = i;
  H->n = n;
  H->wt = NULL;
  H->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  H->off[0] = 0;
  for (i = 0; i < n; i++) {
    for (e = G->off[S[i]]; e < G->off[S[i] + 1]; e++)
      if (pos[G->adj[e]] >= 0) cnt++;
    H->off[i + 1] = cnt;
  }
  H->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cnt > 0 ? cnt : 1));
  cnt = 0;
  for (i = 0; i < n; i++)
    for (e = G->off[S[i]]; e < G->off[S[i] + 1]; e++)
      if (pos[G->adj[e]] >= 0) H->adj[cnt++] = pos[G->adj[e]];
  for (i = 0; i < n; i++) pos[S[i]] = -1;
}

/* A local graph from an edge list (both directions, self-loops dropped,
 * repeated edges kept as separate entries, optional weights). */
static void lgraph_from_edges(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                              const int64_t *w, lgraph *H) {
  int64_t i, *fill;
  H->n = (int32_t)n;
  H->off = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
  for (i = 0; i < m; i++) {
    if (eu[i] == ev[i]) continue;
    H->off[eu[i] + 1]++;
    H->off[ev[i] + 1]++;
  }
  for (i = 0; i < n; i++) H->off[i + 1] += H->off[i];
  H->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(H->off[n] > 0 ? H->off[n] : 1));
  H->wt = w ? (int64_t *)malloc(sizeof(int64_t) * (size_t)(H->off[n] > 0 ? H->off[n] : 1)) : NULL;
  fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  for (i = 0; i <= n; i++) fill[i] = H->off[i];
  for (i = 0; i < m; i++) {
    if (eu[i] == ev[i]) continue;
    if (w) { H->wt[fill[eu[i]]] = w[i]; H->wt[fill[ev[i]]] = w[i]; }
    H->adj[fill[eu[i]]++] = ev[i];
    H->adj[fill[ev[i]]++] = eu[i];
  }
  free(fill);
}

/* ------------------------------------------------------------------------ */
/* GetConnectedComponents (Algorithm 1): breadth-first search started from
 * each unvisited vertex in ascending order, so comp[v] is the smallest id of
 * v's component.  Vertices with alive[v] == 0 are ignored (comp = -1). */
static int32_t components(const lgraph *H, const uint8_t *alive, int32_t *comp) {
  int32_t n = H->n, s, ncomp = 0;
  int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (s = 0; s < n; s++) comp[s] = -1;
  for (s = 0; s < n; s++) {
    int32_t head = 0, tail = 0;
    if ((alive && !alive[s]) || comp[s] >= 0) continue;
    ncomp++;
    comp[s] = s;
    q[tail++] = s;
    while (head < tail) {
      int32_t v = q[head++];
      int64_t e;
      for (e = H->off[v]; e < H->off[v + 1]; e++) {
        int32_t u = H->adj[e];
        if ((alive && !alive[u]) || comp[u] >= 0) continue;
        comp[u] = s;
        q[tail++] = u;
      }
    }
  }
  free(q);
  return ncomp;
}

/* Peeling (not in the paper; required on this path): every round removes, all
 * at once, each alive vertex whose number of alive neighbours is <= T(n) for
 * the current alive count n, until a round removes nothing.  A vertex of
 * degree <= T alone is a cut of value <= T, so the cluster would fail anyway
 * and the singleton side would be dropped.  Returns the alive count. */
static int32_t peel(const lgraph *H, uint8_t *alive, int32_t kind, int64_t num, int64_t den) {
  int32_t n = H->n, i, nalive = 0;
  int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  uint8_t *rem = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
  for (i = 0; i < n; i++) nalive += alive[i] ? 1 : 0;
  for (;;) {
    int64_t T = wo_threshold(kind, num, den, nalive);
    int any = 0;
    for (i = 0; i < n; i++) {
      int64_t e;
      deg[i] = 0;
      if (!alive[i]) continue;
      for (e = H->off[i]; e < H->off[i + 1]; e++) deg[i] += alive[H->adj[e]] ? 1 : 0;
    }
    for (i = 0; i < n; i++) {
      rem[i] = (uint8_t)(alive[i] && deg[i] <= T);
      any |= rem[i];
    }
    if (!any) break;
    for (i = 0; i < n; i++)
      if (rem[i]) { alive[i] = 0; nalive--; }
  }
  free(deg);
  free(rem);
  return nalive;
}

/* ------------------------------------------------------------------------ */
/* Union-find whose root is always the smallest id of its set. */
static int32_t uf_find(int32_t *p, int32_t x) {
  while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
  return x;
}
static void uf_union(int32_t *p, int32_t a, int32_t b) {
  a = uf_find(p, a);
  b = uf_find(p, b);
  if (a < b) p[b] = a;
  else if (b < a) p[a] = b;
}

/* Index of the super-vertex to add next in a maximum-adjacency ordering:
 * among super-vertices X (grp[X] == X) not yet added, the largest key, ties
 * to the smallest id (an ascending scan that only moves on a strictly larger
 * key). */
static int32_t ma_pick(int32_t n, const int32_t *grp, const uint8_t *inA, const int64_t *key) {
  int32_t X = -1, Y;
  for (Y = 0; Y < n; Y++)
    if (grp[Y] == Y && !inA[Y] && (X < 0 || key[Y] > key[X])) X = Y;
  return X;
}

/* Nagamochi-Ibaraki contraction with threshold k (the sparse-certificate
 * step of the exact min cut, GetMinCut in Algorithm 3).  One pass is a
 * maximum-adjacency ordering of the current contracted graph, started from
 * the super-vertex holding local 0, with each key r(Y) = min(w(A, Y), k).
 * When super-vertex X is added, every not-yet-added neighbour Y gets
 * r(Y) <- min(r(Y) + w(X, Y), k); if that value is k, the edge X-Y has
 * q(e) >= k, so X and Y are k-edge-connected and merging them keeps every
 * cut of value < k.  All such pairs are merged after the pass (super-vertex
 * id = smallest local id).  Passes repeat until one super-vertex is left or a
 * pass merges nothing.  rep[v] receives v's super-vertex.  Returns the number
 * of super-vertices left. */
static int32_t ni_contract(const lgraph *H, int64_t k, int32_t *rep, wo_stats *st) {
  int32_t n = H->n, i, nsv = n;
  int64_t *key = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *wadd = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  uint8_t *inA = (uint8_t *)malloc((size_t)n);
  int32_t *uf = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  for (i = 0; i < n; i++) rep[i] = i;
  for (;;) {
    int32_t step, contracted = 0;
    nsv = 0;
    for (i = 0; i < n; i++) nsv += (rep[i] == i);
    if (nsv <= 1) break;
    st->ni_passes++;
    for (i = 0; i < n; i++) { key[i] = 0; wadd[i] = 0; inA[i] = 0; uf[i] = i; }
    for (step = 0; step < nsv; step++) {
      int32_t X = ma_pick(n, rep, inA, key), nt = 0, j;
      inA[X] = 1;
      for (i = 0; i < n; i++) {
        int64_t e;
        if (rep[i] != X) continue;
        for (e = H->off[i]; e < H->off[i + 1]; e++) {
          int32_t Y = rep[H->adj[e]];
          if (Y == X || inA[Y]) continue;
          if (wadd[Y] == 0) touched[nt++] = Y;
          wadd[Y] += H->wt ? H->wt[e] : 1;
        }
      }
      for (j = 0; j < nt; j++) {
        int32_t Y = touched[j];
        key[Y] = key[Y] + wadd[Y] < k ? key[Y] + wadd[Y] : k;
        wadd[Y] = 0;
        if (key[Y] >= k) { uf_union(uf, X, Y); contracted = 1; }
      }
    }
    if (!contracted) break;
    for (i = 0; i < n; i++) rep[i] = uf_find(uf, rep[i]);
  }
  nsv = 0;
  for (i = 0; i < n; i++) nsv += (rep[i] == i);
  free(key); free(wadd); free(inA); free(uf); free(touched);
  return nsv;
}

/* Stoer-Wagner (GetMinCut / MinCutPartition of Algorithm 3) on the graph
 * whose vertices are the groups of grp (grp[v] = smallest local id of v's
 * group), with the canonical tie rule: each phase is a maximum-adjacency
 * ordering with exact (uncapped) keys started from the super-vertex holding
 * local 0, ties to the smallest id; the cut of the phase is the key of the
 * last-added super-vertex t; the minimum is updated only on a strictly
 * smaller cut (earliest phase kept) and its side is t's members; then t and
 * the one added before it, s, are merged.  side[v] = 1 on the kept side.
 * Returns the min cut value. */
static int64_t stoer_wagner(const lgraph *H, int32_t *grp, uint8_t *side, wo_stats *st) {
  int32_t n = H->n, i, nsv = 0;
  int64_t best = INT64_MAX;
  int64_t *key = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  uint8_t *inA = (uint8_t *)malloc((size_t)n);
  for (i = 0; i < n; i++) { nsv += (grp[i] == i); side[i] = 0; }
  while (nsv > 1) {
    int32_t step, s = -1, t = -1, lo, hi;
    int64_t cut = 0;
    st->sw_phases++;
    for (i = 0; i < n; i++) { key[i] = 0; inA[i] = 0; }
    for (step = 0; step < nsv; step++) {
      int32_t X = ma_pick(n, grp, inA, key);
      inA[X] = 1;
      s = t;
      t = X;
      cut = key[X];
      for (i = 0; i < n; i++) {
        int64_t e;
        if (grp[i] != X) continue;
        for (e = H->off[i]; e < H->off[i + 1]; e++) {
          int32_t Y = grp[H->adj[e]];
          if (Y != X && !inA[Y]) key[Y] += H->wt ? H->wt[e] : 1;
        }
      }
    }
    if (cut < best) {
      best = cut;
      for (i = 0; i < n; i++) side[i] = (uint8_t)(grp[i] == t);
    }
    lo = s < t ? s : t;
    hi = s < t ? t : s;
    for (i = 0; i < n; i++)
      if (grp[i] == hi) grp[i] = lo;
    nsv--;
  }
  free(key);
  free(inA);
  return best;
}

/* The cut step of one item (Algorithm 3, lines computing cut and criterion):
 * accept iff the min cut exceeds T.  Returns 1 accept, 0 fail (lambda and
 * side filled), -2 on an internal contradiction. */
static int item_cut(const lgraph *H, int64_t T, int32_t *rep, uint8_t *side, int64_t *lambda,
                    wo_stats *st) {
  int32_t nsv = ni_contract(H, T + 1, rep, st);
  int32_t *grp;
  int64_t lam;
  int32_t i;
  if (nsv == 1) return 1;
  grp = (int32_t *)malloc(sizeof(int32_t) * (size_t)H->n);
  for (i = 0; i < H->n; i++) grp[i] = rep[i];
  lam = stoer_wagner(H, grp, side, st);
  free(grp);
  *lambda = lam;
  /* the contraction stops only after a pass whose last vertex has key < k */
  return lam <= T ? 0 : -2;
}

/* ------------------------------------------------------------------------ */
/* Exported single-step entry points used by the pins. */

int64_t wo_components(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                      int32_t *comp) {
  lgraph H;
  int64_t c;
  lgraph_from_edges(n, m, eu, ev, NULL, &H);
  c = components(&H, NULL, comp);
  lgraph_free(&H);
  return c;
}

int64_t wo_peel(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                int32_t kind, int64_t num, int64_t den, uint8_t *alive) {
  lgraph H;
  int64_t i, r;
  lgraph_from_edges(n, m, eu, ev, NULL, &H);
  for (i = 0; i < n; i++) alive[i] = 1;
  r = peel(&H, alive, kind, num, den);
  lgraph_free(&H);
  return r;
}

int64_t wo_stoer_wagner(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                        const int64_t *w, uint8_t *side) {
  lgraph H;
  wo_stats st;
  int32_t *grp;
  int64_t i, lam;
  if (n < 2) return -1;
  memset(&st, 0, sizeof(st));
  lgraph_from_edges(n, m, eu, ev, w, &H);
  grp = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  for (i = 0; i < n; i++) grp[i] = (int32_t)i;
  lam = stoer_wagner(&H, grp, side, &st);
  free(grp);
  lgraph_free(&H);
  return lam;
}

int wo_item_cut(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev, int64_t T,
                int32_t *rep, uint8_t *side, int64_t *lambda) {
  lgraph H;
  wo_stats st;
  int r, i;
  if (n < 2 || T < 0) return -1;
  memset(&st, 0, sizeof(st));
  lgraph_from_edges(n, m, eu, ev, NULL, &H);
  for (i = 0; i < n; i++) side[i] = 0;
  *lambda = -1;
  r = item_cut(&H, T, rep, side, lambda, &st);
  lgraph_free(&H);
  return r;
}

/* ------------------------------------------------------------------------ */
/* Whole refinement. */

typedef struct {
  int32_t *v; /* ascending global ids */
  int32_t n;
} vset;

typedef struct {
  vset *a;
  int64_t len, cap;
} vlist;

static void vlist_push(vlist *L, const int32_t *v, int32_t n) {
  if (L->len == L->cap) {
    L->cap = L->cap ? 2 * L->cap : 64;
    L->a = (vset *)realloc(L->a, sizeof(vset) * (size_t)L->cap);
  }
  L->a[L->len].v = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  memcpy(L->a[L->len].v, v, sizeof(int32_t) * (size_t)n);
  L->a[L->len].n = n;
  L->len++;
}

/* Push every component of (H, comp) with at least min_size members, each as
 * its ascending list of global ids (S maps local to global). */
static void push_components(vlist *Q, const int32_t *S, const int32_t *comp, int32_t n,
                            int32_t min_size) {
  int32_t i, *cnt, *start, *buf, *fill;
  cnt = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
  start = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  fill = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  buf = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  for (i = 0; i < n; i++)
    if (comp[i] >= 0) cnt[comp[i]]++;
  start[0] = 0;
  for (i = 0; i < n; i++) start[i + 1] = start[i] + cnt[i];
  for (i = 0; i < n; i++) fill[i] = start[i];
  for (i = 0; i < n; i++)
    if (comp[i] >= 0) buf[fill[comp[i]]++] = S[i];
  for (i = 0; i < n; i++)
    if (comp[i] == i && cnt[i] >= min_size) vlist_push(Q, buf + start[i], cnt[i]);
  free(cnt); free(start); free(fill); free(buf);
}

typedef struct {
  int32_t label, v;
} lv_pair;

static int cmp_lv(const void *a, const void *b) {
  const lv_pair *x = (const lv_pair *)a, *y = (const lv_pair *)b;
  if (x->label != y->label) return (x->label > y->label) - (x->label < y->label);
  return (x->v > y->v) - (x->v < y->v);
}

static int cmp_vset_min(const void *a, const void *b) {
  const vset *x = (const vset *)a, *y = (const vset *)b;
  return (x->v[0] > y->v[0]) - (x->v[0] < y->v[0]);
}

/* ------------------------------------------------------------------------ */
/* GetCommunities (Algorithm 5) with a CPM community detection step.  The
 * Constant Potts Model scores a partition P of the part's vertices as
 *   Q(P) = sum over communities c of [ e_c - gamma * n_c (n_c - 1) / 2 ],
 * e_c the edges inside c, n_c its size, gamma = gnum / gden (Section 3 runs
 * Leiden with this quality).  Local moving from singletons: sweeps over the
 * vertices in ascending local id, at most CPM_MAX_SWEEPS of them, stopping
 * after a sweep that moves nothing.  For vertex v, taken out of its
 * community c0, joining community c gains (scaled by gden)
 *   g(c) = k(v, c) * gden - gnum * n_c,
 * k(v, c) = edges from v into c and n_c counted without v; joining an
 * empty community gains 0.  The candidates are the communities of v's
 * neighbours other than c0 and, when c0 holds more than v, an empty
 * community: the id n + v when nobody holds it, else the smallest id nobody
 * holds (community ids are 0..2n-1, at most n of them held; v starts in v;
 * n + v is held when v moved there and others joined it).  The
 * best candidate has the largest gain, ties to the smallest community id; v
 * moves there only when that gain is strictly above g(c0), so every move
 * raises Q and the sweeps end.  Finally (connected != 0, as CM uses it)
 * every community is split into its connected parts (edges inside the
 * community), so that every community handed on is connected.  comm[v] =
 * smallest local id of v's final community.  Returns the number of
 * communities. */
#define CPM_MAX_SWEEPS 64

static int32_t cpm_communities(const lgraph *H, int64_t gnum, int64_t gden, int32_t connected,
                               int32_t *comm) {
  const int32_t n = H->n;
  int32_t *c = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  int64_t *size = (int64_t *)calloc(2 * (size_t)n + 1, sizeof(int64_t));
  int64_t *k = (int64_t *)calloc(2 * (size_t)n + 1, sizeof(int64_t));
  int32_t i, v, sweep, count;
  int64_t q;
  for (v = 0; v < n; v++) {
    c[v] = v;
    size[v] = 1;
  }
  for (sweep = 0; sweep < CPM_MAX_SWEEPS; sweep++) {
    int32_t moved = 0;
    for (v = 0; v < n; v++) {
      const int32_t c0 = c[v];
      int32_t best = -1;
      int64_t bestg = 0, g0;
      for (q = H->off[v]; q < H->off[v + 1]; q++) k[c[H->adj[q]]]++;
      size[c0]--; /* v taken out of c0 */
      g0 = k[c0] * gden - gnum * size[c0];
      for (q = H->off[v]; q < H->off[v + 1]; q++) {
        const int32_t cu = c[H->adj[q]];
        int64_t g;
        if (cu == c0) continue;
        g = k[cu] * gden - gnum * size[cu];
        if (best < 0 || g > bestg || (g == bestg && cu < best)) {
          best = cu;
          bestg = g;
        }
      }
      if (size[c0] > 0) { /* an empty community: n + v, else the smallest empty id */
        int32_t ce = n + v;
        if (size[ce] != 0)
          for (ce = 0; size[ce] != 0; ce++) {
          }
        if (best < 0 || 0 > bestg || (0 == bestg && ce < best)) {
          best = ce;
          bestg = 0;
        }
      }
      for (q = H->off[v]; q < H->off[v + 1]; q++) k[c[H->adj[q]]] = 0;
      if (best >= 0 && bestg > g0) {
        c[v] = best;
        size[best]++;
        moved++;
      } else {
        size[c0]++;
      }
    }
    if (moved == 0) break;
  }
  /* connected parts of every community: union-find over the edges inside
   * a community, root = smallest local id */
  for (v = 0; v < n; v++) comm[v] = v;
  for (v = 0; v < n; v++) {
    if (!connected) { /* the local-moving communities themselves */
      for (i = v + 1; i < n; i++)
        if (c[i] == c[v]) uf_union(comm, i, v);
      continue;
    }
    for (q = H->off[v]; q < H->off[v + 1]; q++) {
      const int32_t u = H->adj[q];
      if (c[u] == c[v]) uf_union(comm, u, v);
    }
  }
  count = 0;
  for (i = 0; i < n; i++) {
    comm[i] = uf_find(comm, i);
    count += comm[i] == i;
  }
  free(c); free(size); free(k);
  return count;
}

/* One work item (Algorithm 3, with the peel and the connectivity check in
 * front of the cut): S is connected-or-not, ascending. */
static int process_item(const graph *G, const int32_t *S, int32_t n, int32_t *pos,
                        int32_t kind, int64_t num, int64_t den, int32_t min_size, int32_t cm,
                        int64_t gnum, int64_t gden, vlist *Q, vlist *W, wo_stats *st) {
  lgraph H, H1;
  uint8_t *alive, *side;
  int32_t *S1, *comp, *rep, *part0, *part1;
  int32_t i, na, nc, n0, n1;
  int64_t T, lam = -1;
  int r, rc = 0;

  st->items++;
  induce(G, S, n, pos, &H);
  alive = (uint8_t *)malloc((size_t)n);
  for (i = 0; i < n; i++) alive[i] = 1;
  na = peel(&H, alive, kind, num, den);
  st->peeled += n - na;
  lgraph_free(&H);
  if (na < min_size) { free(alive); return 0; }

  S1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)na);
  na = 0;
  for (i = 0; i < n; i++)
    if (alive[i]) S1[na++] = S[i];
  free(alive);
  induce(G, S1, na, pos, &H1);

  comp = (int32_t *)malloc(sizeof(int32_t) * (size_t)na);
  nc = components(&H1, NULL, comp);
  if (nc > 1) {
    push_components(Q, S1, comp, na, min_size);
    free(comp); free(S1); lgraph_free(&H1);
    return 0;
  }
  free(comp);

  T = wo_threshold(kind, num, den, na);
  rep = (int32_t *)malloc(sizeof(int32_t) * (size_t)na);
  side = (uint8_t *)malloc((size_t)na);
  r = item_cut(&H1, T, rep, side, &lam, st);
  if (r == 1) {
    vlist_push(W, S1, na); /* Algorithm 3: save V_c */
  } else if (r == 0) {
    /* Algorithm 3: bisect on the min cut and recurse on parts > s_post */
    st->splits++;
    part0 = (int32_t *)malloc(sizeof(int32_t) * (size_t)na);
    part1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)na);
    n0 = n1 = 0;
    for (i = 0; i < na; i++) {
      if (side[i]) part1[n1++] = S1[i];
      else part0[n0++] = S1[i];
    }
    if (!cm) {
      if (n0 >= min_size) vlist_push(Q, part0, n0);
      if (n1 >= min_size) vlist_push(Q, part1, n1);
    } else {
      /* CMC (Algorithm 5): each part above s_post goes through
       * GetCommunities, and every community above s_post is checked again
       * (one community is the whole part, checked again as one unit) */
      int32_t p;
      for (p = 0; p < 2; p++) {
        const int32_t *P = p ? part1 : part0;
        const int32_t np_ = p ? n1 : n0;
        lgraph HP;
        int32_t *cm_comm;
        if (np_ < min_size) continue;
        induce(G, P, np_, pos, &HP);
        cm_comm = (int32_t *)malloc(sizeof(int32_t) * (size_t)np_);
        cpm_communities(&HP, gnum, gden, 1, cm_comm);
        push_components(Q, P, cm_comm, np_, min_size);
        free(cm_comm);
        lgraph_free(&HP);
      }
    }
    free(part0); free(part1);
  } else {
    rc = -2;
  }
  free(rep); free(side); free(S1);
  lgraph_free(&H1);
  return rc;
}

static int refine_all(int64_t n, const int64_t *off, const int32_t *adj, const int32_t *label_in,
                      int32_t kind, int64_t num, int64_t den, int32_t min_size, int32_t cm,
                      int64_t gnum, int64_t gden, const uint8_t *only_label, int64_t n_only,
                      int32_t out_mode, int32_t *label_out, wo_stats *stats) {
  graph G;
  wo_stats st;
  lv_pair *pairs;
  int32_t *pos, *S, *comp;
  int64_t v, np = 0, i, j;
  vlist Q = {0, 0, 0}, W = {0, 0, 0};
  int rc = 0;

  if (n < 0 || n > INT32_MAX) return -1;
  if (wo_threshold(kind, num, den, 1) < 0) return -1;
  memset(&st, 0, sizeof(st));
  if (min_size < 2) min_size = 2; /* a singleton has no edge and is never saved */
  G.n = n; G.off = off; G.adj = adj;

  /* group the clustered vertices by input label, ascending id within a group */
  pairs = (lv_pair *)malloc(sizeof(lv_pair) * (size_t)(n > 0 ? n : 1));
  for (v = 0; v < n; v++) {
    int32_t c = label_in[v];
    if (c < 0) continue;
    if (only_label && (c >= n_only || !only_label[c])) continue;
    pairs[np].label = c;
    pairs[np].v = (int32_t)v;
    np++;
  }
  qsort(pairs, (size_t)np, sizeof(lv_pair), cmp_lv);

  pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (v = 0; v < n; v++) pos[v] = -1;
  S = (int32_t *)malloc(sizeof(int32_t) * (size_t)(np > 0 ? np : 1));
  comp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(np > 0 ? np : 1));

  /* CCR (Algorithm 1): every input cluster is split into its connected
   * components and each component with at least min_size vertices queued */
  for (i = 0; i < np; i = j) {
    lgraph H;
    int32_t cn = 0;
    for (j = i; j < np && pairs[j].label == pairs[i].label; j++) S[cn++] = pairs[j].v;
    st.in_clusters++;
    induce(&G, S, cn, pos, &H);
    components(&H, NULL, comp);
    push_components(&Q, S, comp, cn, min_size);
    lgraph_free(&H);
  }

  /* WCC (Algorithm 2) / isWCC (Algorithm 3): drain the queue */
  while (Q.len > 0 && rc == 0) {
    vset it = Q.a[--Q.len];
    rc = process_item(&G, it.v, it.n, pos, kind, num, den, min_size, cm, gnum, gden, &Q, &W,
                      &st);
    free(it.v);
  }

  /* unique cluster identifiers: ascending smallest vertex id */
  for (v = 0; v < n; v++) label_out[v] = -1;
  qsort(W.a, (size_t)W.len, sizeof(vset), cmp_vset_min);
  for (i = 0; i < W.len; i++)
    for (j = 0; j < W.a[i].n; j++)
      label_out[W.a[i].v[j]] = out_mode == 1 ? W.a[i].v[0] : (int32_t)i;
  st.out_clusters = W.len;

  for (i = 0; i < W.len; i++) free(W.a[i].v);
  for (i = 0; i < Q.len; i++) free(Q.a[i].v);
  free(W.a); free(Q.a);
  free(pairs); free(pos); free(S); free(comp);
  if (stats) *stats = st;
  return rc;
}

int wo_wcc(int64_t n, const int64_t *off, const int32_t *adj, const int32_t *label_in,
           int32_t kind, int64_t num, int64_t den, int32_t min_size,
           const uint8_t *only_label, int64_t n_only, int32_t out_mode,
           int32_t *label_out, wo_stats *stats) {
  return refine_all(n, off, adj, label_in, kind, num, den, min_size, 0, 0, 1, only_label, n_only,
                    out_mode, label_out, stats);
}

/* CM (Section 2.4, Algorithms 4-5): WCC whose split parts go through the CPM
 * community step before they are checked again. */
int wo_cm(int64_t n, const int64_t *off, const int32_t *adj, const int32_t *label_in,
          int32_t kind, int64_t num, int64_t den, int32_t min_size, int64_t gnum, int64_t gden,
          const uint8_t *only_label, int64_t n_only, int32_t out_mode, int32_t *label_out,
          wo_stats *stats) {
  if (gnum < 0 || gden < 1) return -1;
  return refine_all(n, off, adj, label_in, kind, num, den, min_size, 1, gnum, gden, only_label,
                    n_only, out_mode, label_out, stats);
}

int64_t wo_cpm_communities(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                           int64_t gnum, int64_t gden, int32_t connected, int32_t *comm) {
  lgraph H;
  int64_t r;
  if (n < 0 || gnum < 0 || gden < 1) return -1;
  lgraph_from_edges(n, m, eu, ev, NULL, &H);
  r = cpm_communities(&H, gnum, gden, connected, comm);
  lgraph_free(&H);
  return r;
}
