// Oracle: a plain, slow, single-threaded CPU statement of the patch-guided
// nested-dissection ordering of "Fast Sparse Matrix Permutation for Mesh-Based
// Direct Solvers" (Algorithm 1 overview; Algorithm 2 GetSeparator; Algorithm 3
// ComputePerm; Sections 4.1-4.3 and 5) together with the textbook symbolic
// Cholesky quantities (elimination tree, column counts).
//
// TEST INFRASTRUCTURE ONLY. Nothing in the library links or calls this file;
// only the tests, the smoke check and the benchmark's CPU-baseline leg do.
// It shares no code, header, table or constant generator with the CUDA path.
//
// Where the paper leaves a choice open (its patcher, the METIS bisection and
// node refinement, AMD) this file follows the deterministic readings of the
// determinism contract, each restated at the function that implements it.
// Readability over speed: plain std::vector / std::set / std::map, no
// blocking, no fusion, no reordering beyond what a definition states.
//
// Parity status: every function below is pinned by a CPU test against
// brute force, a closed form or an invariant, except where its header says
// "parity unpinned".

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <vector>

namespace {

typedef std::vector<std::vector<int32_t>> Adj;   // sorted neighbour lists

const int32_t INF = INT32_MAX;

// SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): the output for generator state `s` is the
// finaliser applied to s + gamma.
uint64_t splitmix64_at(uint64_t s) {
  uint64_t z = s + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Contract R1: the seed hash h(v) = SplitMix64 at state seed*gamma + v.
uint64_t seed_hash(uint64_t seed, int32_t v) {
  return splitmix64_at(seed * 0x9E3779B97F4A7C15ULL + (uint64_t)(uint32_t)v);
}

// Contract R9: the tie-break hash of a vertex for separator refinement.
uint32_t tie_hash(int32_t v) {
  return (uint32_t)(splitmix64_at((uint64_t)(uint32_t)v) >> 32);
}

// ---------------------------------------------------------------------------
// Section 2 / Section 4.1 step 2: G is the graph of A without its diagonal.
// ---------------------------------------------------------------------------

// Undirected simple graph of a face list: {a,b} is an edge iff a and b are
// consecutive corners of some face and a != b.
bool graph_from_faces(const int32_t* faces, int64_t nf, int32_t n, Adj& adj) {
  adj.assign(n, {});
  for (int64_t f = 0; f < nf; ++f) {
    for (int c = 0; c < 3; ++c) {
      int32_t a = faces[3 * f + c], b = faces[3 * f + (c + 1) % 3];
      if (a < 0 || a >= n || b < 0 || b >= n) return false;
      if (a == b) continue;
      adj[a].push_back(b);
      adj[b].push_back(a);
    }
  }
  for (auto& r : adj) {
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
  }
  return true;
}

// Graph of a (scalar or b x b block) symmetric pattern, Section 4.1 step 2 and
// Section 6.5: each b x b block is merged into one vertex; vertices u != v are
// adjacent iff some entry of block (u, v) is present. Returns 0 ok, -1 bad
// index, -2 not structurally symmetric.
int graph_from_pattern(const int32_t* rowptr, const int32_t* col, int32_t nrows, int32_t b, Adj& adj) {
  if (b < 1 || nrows % b != 0) return -1;
  int32_t n = nrows / b;
  adj.assign(n, {});
  for (int32_t i = 0; i < nrows; ++i)
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int32_t j = col[e];
      if (j < 0 || j >= nrows) return -1;
      if (i / b != j / b) adj[i / b].push_back(j / b);
    }
  for (auto& r : adj) {
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
  }
  for (int32_t u = 0; u < n; ++u)
    for (int32_t v : adj[u])
      if (!std::binary_search(adj[v].begin(), adj[v].end(), u)) return -2;
  return 0;
}

// ---------------------------------------------------------------------------
// Section 4.1 step 1, GetPatches (Algorithm 1). The paper uses RXMesh's GPU
// Lloyd patcher; the contract replaces it by seeded BFS Voronoi cells,
// R Lloyd re-centring rounds and a hard size cap.
// ---------------------------------------------------------------------------

// Contract R2: multi-source BFS Voronoi labelling. dist(v) is the hop distance
// to the nearest source along allowed edges; label(v) is the smallest rank
// among the sources at that distance. An edge {u,v} is allowed iff group is
// null or group[u] == group[v]. Stated level by level: a vertex first reached
// at level d takes the minimum label over its neighbours at level d-1.
// Vertices not reached keep dist INF / label -1.
void voronoi(const Adj& adj, const std::vector<int32_t>& src, const std::vector<int32_t>& rank,
             const int32_t* group, std::vector<int32_t>& dist, std::vector<int32_t>& label) {
  std::vector<int32_t> frontier;
  for (size_t i = 0; i < src.size(); ++i) {
    dist[src[i]] = 0;
    label[src[i]] = rank[i];
    frontier.push_back(src[i]);
  }
  for (int32_t d = 0; !frontier.empty(); ++d) {
    std::vector<int32_t> next;
    for (int32_t u : frontier)
      for (int32_t v : adj[u]) {
        if (group && group[u] != group[v]) continue;
        if (dist[v] == INF) {
          dist[v] = d + 1;
          label[v] = label[u];
          next.push_back(v);
        } else if (dist[v] == d + 1) {
          label[v] = std::min(label[v], label[u]);
        }
      }
    frontier.swap(next);
  }
}

// Contract R1: v is a seed iff (h(v) >> 32) * n < k_target * 2^32 with
// k_target = max(1, ceil(2n / cap)) (the paper's target patch size is read as
// a mean of cap/2, Section 6). Seeds are ranked in increasing vertex id.
void select_seeds(int32_t n, int32_t cap, uint64_t seed, std::vector<int32_t>& seeds) {
  uint64_t kt = ((uint64_t)2 * (uint64_t)n + (uint64_t)cap - 1) / (uint64_t)cap;
  if (kt < 1) kt = 1;
  for (int32_t v = 0; v < n; ++v) {
    uint64_t u = seed_hash(seed, v) >> 32;
    if (u * (uint64_t)n < (kt << 32)) seeds.push_back(v);
  }
}

struct Patching {
  std::vector<int32_t> label;        // patch id (= rank) per vertex
  std::vector<int32_t> seed_of;      // seed vertex per rank
  int32_t k = 0;
};

// What the patching stage passes through, for tests that check each step
// (and the library's stage dump) rather than only the final labels.
struct PatchTrace {
  std::vector<int32_t> seeds0;                     // seed of every rank after R1 + R3
  std::vector<std::vector<int32_t>> lloyd_seeds;   // seed of every rank after each Lloyd round
  std::vector<std::vector<int32_t>> labels;        // labels after the first labelling and each Lloyd relabel
};

// Patching from given seeds (rank = position in `seeds`): Voronoi cells,
// unreached components, R Lloyd rounds, cap splitting (contract R2-R5).
Patching patches_from_seeds(const Adj& adj, const std::vector<int32_t>& seeds, int32_t cap, int32_t lloyd_rounds,
                            PatchTrace* tr) {
  int32_t n = (int32_t)adj.size();
  Patching P;
  P.label.assign(n, -1);
  std::vector<int32_t> dist(n, INF);
  P.seed_of = seeds;
  std::vector<int32_t> ranks(P.seed_of.size());
  for (size_t r = 0; r < ranks.size(); ++r) ranks[r] = (int32_t)r;
  voronoi(adj, P.seed_of, ranks, nullptr, dist, P.label);

  // R3: each connected component that no seed reached gets its smallest
  // vertex id as a new seed; new ranks follow in increasing vertex id.
  {
    std::vector<int32_t> extra;
    std::vector<char> seen(n, 0);
    for (int32_t v = 0; v < n; ++v) {
      if (P.label[v] != -1 || seen[v]) continue;
      extra.push_back(v);
      std::vector<int32_t> stack = {v};
      seen[v] = 1;
      while (!stack.empty()) {
        int32_t u = stack.back(); stack.pop_back();
        for (int32_t w : adj[u]) if (!seen[w]) { seen[w] = 1; stack.push_back(w); }
      }
    }
    if (!extra.empty()) {
      std::vector<int32_t> xr;
      for (int32_t v : extra) { xr.push_back((int32_t)P.seed_of.size()); P.seed_of.push_back(v); }
      voronoi(adj, extra, xr, nullptr, dist, P.label);
    }
  }
  P.k = (int32_t)P.seed_of.size();
  if (tr) { tr->seeds0 = P.seed_of; tr->labels.push_back(P.label); }

  // R4 Lloyd rounds: the new seed of a patch is its vertex farthest (in hops
  // inside the patch) from the patch boundary, ties to the lowest id; a patch
  // without boundary keeps its seed. Then every vertex is relabelled.
  for (int32_t it = 0; it < lloyd_rounds; ++it) {
    std::vector<int32_t> bsrc, bzero;
    for (int32_t v = 0; v < n; ++v)
      for (int32_t u : adj[v])
        if (P.label[u] != P.label[v]) { bsrc.push_back(v); bzero.push_back(0); break; }
    std::vector<int32_t> depth(n, INF), dummy(n, -1);
    voronoi(adj, bsrc, bzero, P.label.data(), depth, dummy);
    std::vector<int32_t> best(P.k, -1);
    for (int32_t v = 0; v < n; ++v) {
      if (depth[v] == INF) continue;
      int32_t p = P.label[v];
      if (best[p] == -1 || depth[v] > depth[best[p]] || (depth[v] == depth[best[p]] && v < best[p])) best[p] = v;
    }
    for (int32_t p = 0; p < P.k; ++p) if (best[p] != -1) P.seed_of[p] = best[p];
    std::fill(P.label.begin(), P.label.end(), -1);
    std::fill(dist.begin(), dist.end(), INF);
    std::vector<int32_t> all(P.k);
    for (int32_t p = 0; p < P.k; ++p) all[p] = p;
    voronoi(adj, P.seed_of, all, nullptr, dist, P.label);
    if (tr) { tr->lloyd_seeds.push_back(P.seed_of); tr->labels.push_back(P.label); }
  }

  // R5 cap: while some patch is larger than cap, each such patch gets a second
  // seed, its vertex farthest from its seed inside the patch (ties to the
  // lowest id), ranked after all existing ranks in the order of the parent
  // rank; then only that patch is relabelled from its two seeds.
  for (;;) {
    std::vector<int32_t> size(P.k, 0);
    for (int32_t v = 0; v < n; ++v) size[P.label[v]]++;
    std::vector<int32_t> over;
    for (int32_t p = 0; p < P.k; ++p) if (size[p] > cap) over.push_back(p);
    if (over.empty()) break;
    std::vector<int32_t> old = P.label;
    std::vector<int32_t> srcs, srank;
    for (int32_t p : over) { srcs.push_back(P.seed_of[p]); srank.push_back(p); }
    std::vector<int32_t> d(n, INF), dl(n, -1);
    voronoi(adj, srcs, srank, old.data(), d, dl);
    std::vector<int32_t> far(P.k, -1);
    for (int32_t v = 0; v < n; ++v) {
      if (d[v] == INF) continue;
      int32_t p = old[v];
      if (far[p] == -1 || d[v] > d[far[p]] || (d[v] == d[far[p]] && v < far[p])) far[p] = v;
    }
    std::vector<char> is_over(P.k, 0);
    for (int32_t p : over) is_over[p] = 1;
    std::vector<int32_t> s2, r2;
    for (int32_t p : over) {       // increasing parent rank
      int32_t r = (int32_t)P.seed_of.size();
      P.seed_of.push_back(far[p]);
      s2.push_back(P.seed_of[p]); r2.push_back(p);
      s2.push_back(far[p]); r2.push_back(r);
    }
    for (int32_t v = 0; v < n; ++v) if (is_over[old[v]]) { P.label[v] = -1; dist[v] = INF; }
    voronoi(adj, s2, r2, old.data(), dist, P.label);
    P.k = (int32_t)P.seed_of.size();
  }
  return P;
}

// Full patching (contract R1-R5): seeds by the hash rule, then as above.
Patching get_patches(const Adj& adj, int32_t cap, uint64_t seed, int32_t lloyd_rounds, PatchTrace* tr = nullptr) {
  std::vector<int32_t> seeds;
  select_seeds((int32_t)adj.size(), cap, seed, seeds);
  return patches_from_seeds(adj, seeds, cap, lloyd_rounds, tr);
}

// ---------------------------------------------------------------------------
// Section 4.2 BuildEtree with Algorithm 2 GetSeparator, quotient graph built
// once and updated by weight decrements (Section 5, "Quotient graph
// computation").
// ---------------------------------------------------------------------------

int32_t ceil_log2_of(int64_t k) {
  int32_t d = 0;
  while (((int64_t)1 << d) < k) ++d;
  return d;
}

struct NDTree {
  int32_t D = 0;
  std::vector<int32_t> node_of;        // tree node of every vertex
};

struct ND {
  const Adj& adj;
  const std::vector<int32_t>& patch;
  int32_t D;
  std::vector<int32_t> w;                        // R6 node weights
  std::vector<std::map<int32_t, int32_t>> qw;    // R6 edge weights
  std::vector<char> removed;
  std::vector<int32_t> node_of;
  // scratch, reset after each use so that a node costs O(its own size)
  std::vector<char> here, released, newsep, inS, sideS, done;
  std::vector<int32_t> cdeg;
  std::map<int32_t, int64_t> qsum_at;     // node -> sum of w(p,q), p,q in S (trace)
  // stage trace (filled when `trace` is set): per depth d and patch p, the
  // side (0 left, 1 right) p took in the node bisected at depth d, and the
  // child node p moved to (-1 once it has no remaining vertex); -1 where p
  // took part in no bisection at depth d
  bool trace = false;
  std::vector<std::vector<int32_t>> side_at, child_at;

  ND(const Adj& a, const std::vector<int32_t>& p, int32_t k, int32_t d)
      : adj(a), patch(p), D(d), w(k, 0), qw(k), removed(a.size(), 0), node_of(a.size(), -1),
        here(a.size(), 0), released(a.size(), 0), newsep(a.size(), 0), inS(k, 0), sideS(k, 0),
        done(k, 0), cdeg(a.size(), 0) {
    // Quotient graph (Section 3 definition; Algorithm 2 step 1), built once.
    for (size_t v = 0; v < adj.size(); ++v) {
      w[patch[v]]++;
      for (int32_t u : adj[v])
        if (patch[u] != patch[v]) qw[patch[v]][patch[u]]++;
    }
  }

  int32_t qdeg(int32_t p, const std::vector<char>& inS) const {
    int32_t d = 0;
    for (auto& e : qw[p]) if (e.second > 0 && inS[e.first]) ++d;
    return d;
  }

  // BFS levels over the quotient subgraph on S from r (edges of weight > 0).
  std::vector<std::vector<int32_t>> qbfs(int32_t r, const std::vector<char>& inS) const {
    std::vector<std::vector<int32_t>> lv = {{r}};
    std::set<int32_t> seen = {r};
    while (true) {
      std::vector<int32_t> nx;
      for (int32_t p : lv.back())
        for (auto& e : qw[p])
          if (e.second > 0 && inS[e.first] && !seen.count(e.first)) { seen.insert(e.first); nx.push_back(e.first); }
      if (nx.empty()) break;
      lv.push_back(nx);
    }
    return lv;
  }

  // Contract R8, BiPartition (Algorithm 2 step 2; METIS with its balance
  // constraint in the paper, which balances the quotient graph's vertex
  // weights): order S component by component (components by their smallest
  // patch id); inside a component, r0 = min (degree, id), r1 = min (degree,
  // id) on the last BFS level from r0, and the patches are ordered by (BFS
  // level from r1, id). With o_1..o_m that order, W the summed weight w(p) of
  // S and P_j the weight of o_1..o_j, Left = o_1..o_j for the j in J whose
  // |2 P_j - W| is smallest (ties to the smaller j): the cut of the order that
  // best halves the remaining vertices. J keeps each child within the patch
  // capacity of its subtree, so that with the default depth every leaf is a
  // single patch: with D' = min(D, ceil(log2 k)) and c = 2^(D' - depth - 1),
  // J = [max(1, m - c), min(m - 1, c)], or [1, m - 1] when that is empty
  // (only when an explicit depth below ceil(log2 k) makes leaves hold
  // several patches anyway).
  // Returns with sideS[p] set for p in S (0 left, 1 right); inS marks S.
  void bipartition(const std::vector<int32_t>& S, int32_t depth) {
    for (int32_t p : S) { inS[p] = 1; sideS[p] = 0; done[p] = 0; }
    std::vector<int32_t> order;
    std::vector<int32_t> sorted = S;
    std::sort(sorted.begin(), sorted.end());
    for (int32_t c0 : sorted) {
      if (done[c0]) continue;
      auto comp_lv = qbfs(c0, inS);
      int32_t r0 = -1, best = INT32_MAX;
      for (auto& l : comp_lv) for (int32_t p : l) {
        int32_t dg = qdeg(p, inS);
        if (dg < best || (dg == best && p < r0)) { best = dg; r0 = p; }
      }
      auto lv0 = qbfs(r0, inS);
      int32_t r1 = -1; best = INT32_MAX;
      for (int32_t p : lv0.back()) {
        int32_t dg = qdeg(p, inS);
        if (dg < best || (dg == best && p < r1)) { best = dg; r1 = p; }
      }
      auto lv1 = qbfs(r1, inS);
      for (auto& l : lv1) {
        std::vector<int32_t> s = l;
        std::sort(s.begin(), s.end());
        for (int32_t p : s) { order.push_back(p); done[p] = 1; }
      }
    }
    const int64_t m = (int64_t)order.size();
    const int32_t Dp = std::min(D, ceil_log2_of((int64_t)w.size()));
    int64_t lo = 1, hi = m - 1;
    if (Dp - depth - 1 >= 0 && Dp - depth - 1 < 62) {
      const int64_t c = (int64_t)1 << (Dp - depth - 1);
      if (std::max<int64_t>(1, m - c) <= std::min<int64_t>(m - 1, c)) {
        lo = std::max<int64_t>(1, m - c);
        hi = std::min<int64_t>(m - 1, c);
      }
    }
    int64_t W = 0;
    for (int32_t p : order) W += w[p];
    int64_t nl = lo;
    int64_t P = 0, best_gap = INT64_MAX;
    for (int64_t j = 1; j <= hi; ++j) {
      P += w[order[j - 1]];
      if (j < lo) continue;
      const int64_t gap = 2 * P > W ? 2 * P - W : W - 2 * P;
      if (gap < best_gap) { best_gap = gap; nl = j; }
    }
    for (int64_t i = nl; i < m; ++i) sideS[order[i]] = 1;
  }

  void node(int32_t t, int32_t depth, std::vector<int32_t> S, const std::vector<int32_t>& verts) {
    // Patches whose remaining weight is zero take no part (contract R7).
    std::vector<int32_t> S2;
    for (int32_t p : S) if (w[p] > 0) S2.push_back(p);
    S.swap(S2);
    if (depth == D || S.size() <= 1) {           // leaf: stores the remaining vertices
      for (int32_t v : verts) node_of[v] = t;
      return;
    }
    bipartition(S, depth);
    const std::vector<char>& side = sideS;
    if (trace) {
      if ((int32_t)side_at.size() <= depth) {
        side_at.resize(depth + 1, std::vector<int32_t>(w.size(), -1));
        child_at.resize(depth + 1, std::vector<int32_t>(w.size(), -1));
      }
      for (int32_t p : S) side_at[depth][p] = side[p];
    }
    int64_t qs = 0;
    for (int32_t p : S)
      for (auto& e : qw[p]) if (inS[e.first]) qs += e.second;
    qsum_at[t] = qs;
    for (int32_t v : verts) here[v] = 1;

    // Algorithm 2 step 3, SuperSeparator: remaining vertices of this node with
    // a neighbour (also remaining here) on the other side.
    std::vector<int32_t> super;
    for (int32_t v : verts) {
      for (int32_t u : adj[v])
        if (here[u] && side[patch[u]] != side[patch[v]]) cdeg[v]++;
      if (cdeg[v] > 0) super.push_back(v);
    }
    // Algorithm 2 step 4, RefineSeparator (contract R9; METIS node refinement
    // in the paper): greedily release superset vertices back to their side in
    // increasing (cdeg, tie_hash, id), a vertex being released iff none of its
    // crossing neighbours was released before it. The separator is what stays:
    // a minimal vertex cover of the crossing edges.
    std::sort(super.begin(), super.end(), [&](int32_t a, int32_t b) {
      if (cdeg[a] != cdeg[b]) return cdeg[a] < cdeg[b];
      uint32_t ha = tie_hash(a), hb = tie_hash(b);
      if (ha != hb) return ha < hb;
      return a < b;
    });
    for (int32_t v : super) {
      bool ok = true;
      for (int32_t u : adj[v])
        if (here[u] && side[patch[u]] != side[patch[v]] && released[u]) { ok = false; break; }
      if (ok) released[v] = 1;
    }
    for (int32_t v : super) if (!released[v]) { newsep[v] = 1; node_of[v] = t; }

    // Section 5: remove the separator's weight from the quotient graph: node
    // weights lose the separator vertices, edge weights lose every G-edge
    // between two remaining vertices of different patches that touches the
    // separator (each such edge once).
    for (int32_t v : verts) {
      if (!newsep[v]) continue;
      w[patch[v]]--;
      for (int32_t u : adj[v]) {
        if (!here[u] || patch[u] == patch[v]) continue;
        if (newsep[u] && u < v) continue;        // counted from u
        qw[patch[v]][patch[u]]--;
        qw[patch[u]][patch[v]]--;
      }
    }
    for (int32_t v : verts) if (newsep[v]) removed[v] = 1;
    if (trace)
      for (int32_t p : S) child_at[depth][p] = w[p] > 0 ? 2 * t + 1 + side[p] : -1;

    // Algorithm 2 step 5, LeftRight: children 2t+1 (left) and 2t+2 (right).
    std::vector<int32_t> SL, SR, VL, VR;
    for (int32_t p : S) (side[p] ? SR : SL).push_back(p);
    for (int32_t v : verts) if (!newsep[v]) (side[patch[v]] ? VR : VL).push_back(v);
    for (int32_t v : verts) { here[v] = 0; released[v] = 0; newsep[v] = 0; cdeg[v] = 0; }
    for (int32_t p : S) inS[p] = 0;
    node(2 * t + 1, depth + 1, SL, VL);
    node(2 * t + 2, depth + 1, SR, VR);
  }
};

int32_t ceil_log2(int64_t k) {
  int32_t d = 0;
  while (((int64_t)1 << d) < k) ++d;
  return d;
}

// ---------------------------------------------------------------------------
// Algorithm 3 step 1, LocalOrder (AMD in the paper; contract R11 reads it as
// exact minimum degree): repeatedly eliminate the vertex of smallest current
// degree in the elimination graph, ties to the smallest original id, and make
// its neighbours a clique.
// ---------------------------------------------------------------------------
std::vector<int32_t> min_degree(const Adj& adj, const std::vector<int32_t>& verts,
                                const std::vector<uint32_t>* key = nullptr) {
  std::map<int32_t, int32_t> loc;
  for (size_t i = 0; i < verts.size(); ++i) loc[verts[i]] = (int32_t)i;
  std::vector<std::set<int32_t>> g(verts.size());
  for (size_t i = 0; i < verts.size(); ++i)
    for (int32_t u : adj[verts[i]]) {
      auto it = loc.find(u);
      if (it != loc.end()) g[i].insert(it->second);
    }
  std::vector<char> alive(verts.size(), 1);
  std::vector<int32_t> order;
  for (size_t step = 0; step < verts.size(); ++step) {
    int32_t p = -1;
    for (size_t i = 0; i < verts.size(); ++i) {
      if (!alive[i]) continue;
      if (p == -1 || g[i].size() < g[p].size()) { p = (int32_t)i; continue; }
      if (g[i].size() != g[p].size()) continue;
      // equal degrees: the smaller (key, id) wins; without keys, the smaller id
      const uint32_t ki = key ? (*key)[i] : 0u, kp = key ? (*key)[p] : 0u;
      if (ki < kp || (ki == kp && verts[i] < verts[p])) p = (int32_t)i;
    }
    order.push_back(verts[p]);
    alive[p] = 0;
    std::vector<int32_t> nb(g[p].begin(), g[p].end());
    for (int32_t a : nb) {
      g[a].erase(p);
      for (int32_t b : nb) if (b != a) g[a].insert(b);
    }
    g[p].clear();
  }
  return order;
}

// The learned-priority variant (the paper is silent on learned orderings; this
// is the reading used for them): the same exact minimum degree, but a tie
// between equal degrees goes to the smaller (key, original id), key being a
// per-vertex priority (a network score mapped to a key, or a seeded hash).
// With all keys equal it is min_degree above.

// Algorithm 3 step 2 with the two schedules of Section 5: post-order (left
// subtree, right subtree, node) or level order (deepest level first, nodes in
// index order within a level).
void concat_schedule(int32_t t, int32_t nnodes, const std::vector<std::vector<int32_t>>& local,
                     std::vector<int32_t>& perm, std::vector<int32_t>& begin) {
  if (t >= nnodes) return;
  concat_schedule(2 * t + 1, nnodes, local, perm, begin);
  concat_schedule(2 * t + 2, nnodes, local, perm, begin);
  begin[t] = (int32_t)perm.size();
  perm.insert(perm.end(), local[t].begin(), local[t].end());
}

// ---------------------------------------------------------------------------
// Symbolic Cholesky of B = P (G + I) P^T (textbook: Liu 1990; George & Liu):
// parent[j] = min{ i > j : L_ij != 0 } (-1 if none), colcount[j] = |{ i >= j :
// L_ij != 0 }|. The etree follows from the definition via path-compressed
// ancestors; row i of L is the union of the tree paths from each j < i with
// B_ij != 0 up to i, which gives the column counts.
// ---------------------------------------------------------------------------
void symbolic(const Adj& adj, const int32_t* perm, std::vector<int32_t>& parent,
              std::vector<int32_t>& colcount, int64_t& nnzL, int64_t& flops) {
  int32_t n = (int32_t)adj.size();
  std::vector<int32_t> iperm(n);
  for (int32_t i = 0; i < n; ++i) iperm[perm[i]] = i;
  parent.assign(n, -1);
  std::vector<int32_t> anc(n, -1);
  for (int32_t i = 0; i < n; ++i) {
    for (int32_t u : adj[perm[i]]) {
      int32_t j = iperm[u];
      if (j >= i) continue;
      // climb from j to the root of its current subtree, pointing the path at i
      while (j != -1 && j < i) {
        int32_t nx = anc[j];
        anc[j] = i;
        if (nx == -1) parent[j] = i;
        j = nx;
      }
    }
  }
  colcount.assign(n, 1);
  std::vector<int32_t> mark(n, -1);
  for (int32_t i = 0; i < n; ++i) {
    mark[i] = i;
    for (int32_t u : adj[perm[i]]) {
      int32_t j = iperm[u];
      if (j >= i) continue;
      while (mark[j] != i) { colcount[j]++; mark[j] = i; j = parent[j]; }
    }
  }
  nnzL = 0; flops = 0;
  for (int32_t j = 0; j < n; ++j) { nnzL += colcount[j]; flops += (int64_t)colcount[j] * colcount[j]; }
}

Adj adj_from_csr(const int32_t* rowptr, const int32_t* col, int32_t n) {
  Adj a(n);
  for (int32_t i = 0; i < n; ++i) a[i].assign(col + rowptr[i], col + rowptr[i + 1]);
  return a;
}

int64_t adj_to_csr(const Adj& a, int32_t* rowptr, int32_t* col, int64_t cap) {
  int64_t nnz = 0;
  for (auto& r : a) nnz += (int64_t)r.size();
  if (!rowptr) return nnz;
  if (nnz > cap) return -3;
  int64_t e = 0;
  rowptr[0] = 0;
  for (size_t i = 0; i < a.size(); ++i) {
    for (int32_t v : a[i]) col[e++] = v;
    rowptr[i + 1] = (int32_t)e;
  }
  return nnz;
}

}  // namespace

// ===========================================================================
// Flat C interface (ctypes) -- test infrastructure only.
// ===========================================================================
extern "C" {

typedef struct {
  int32_t patch_cap;
  uint64_t seed;
  int32_t lloyd_rounds;
  int32_t nd_level;       // 0 = ceil(log2 k)
  int32_t schedule;       // 0 post-order, 1 level order
} oracle_opts;

// Graph of a face list. With rowptr == NULL returns nnz (2E) only; else fills
// rowptr[n+1], col[nnz]. Returns -1 for an out-of-range corner.
int64_t oracle_graph_from_faces(const int32_t* faces, int64_t nf, int32_t n,
                                int32_t* rowptr, int32_t* col, int64_t cap) {
  Adj a;
  if (!graph_from_faces(faces, nf, n, a)) return -1;
  return adj_to_csr(a, rowptr, col, cap);
}

// Vertex graph of a scalar (b = 1) or block pattern. -1 bad input, -2 not
// structurally symmetric.
int64_t oracle_graph_from_pattern(const int32_t* rowptr, const int32_t* col, int32_t nrows, int32_t b,
                                  int32_t* out_rowptr, int32_t* out_col, int64_t cap) {
  Adj a;
  int rc = graph_from_pattern(rowptr, col, nrows, b, a);
  if (rc) return rc;
  return adj_to_csr(a, out_rowptr, out_col, cap);
}

uint64_t oracle_seed_hash(uint64_t seed, int32_t v) { return seed_hash(seed, v); }

// Seeds in rank order; returns the count (seeds may be NULL to count only).
int32_t oracle_seeds(int32_t n, int32_t cap, uint64_t seed, int32_t* seeds) {
  std::vector<int32_t> s;
  select_seeds(n, cap, seed, s);
  if (seeds) std::copy(s.begin(), s.end(), seeds);
  return (int32_t)s.size();
}

// Voronoi labelling from explicit sources (group may be NULL).
void oracle_voronoi(const int32_t* rowptr, const int32_t* col, int32_t n, int32_t nsrc,
                    const int32_t* src, const int32_t* rank, const int32_t* group,
                    int32_t* dist_out, int32_t* label_out) {
  Adj a = adj_from_csr(rowptr, col, n);
  std::vector<int32_t> s(src, src + nsrc), r(rank, rank + nsrc), d(n, INF), l(n, -1);
  voronoi(a, s, r, group, d, l);
  for (int32_t v = 0; v < n; ++v) { dist_out[v] = d[v] == INF ? -1 : d[v]; label_out[v] = l[v]; }
}

// Patch labels (gmap); returns k.
int32_t oracle_patches(const int32_t* rowptr, const int32_t* col, int32_t n, int32_t cap,
                       uint64_t seed, int32_t lloyd_rounds, int32_t* label) {
  if (cap < 1) return -1;
  Adj a = adj_from_csr(rowptr, col, n);
  Patching P = get_patches(a, cap, seed, lloyd_rounds);
  std::copy(P.label.begin(), P.label.end(), label);
  return P.k;
}

// Exact minimum-degree order of the whole graph.
void oracle_min_degree(const int32_t* rowptr, const int32_t* col, int32_t n, int32_t* order) {
  Adj a = adj_from_csr(rowptr, col, n);
  std::vector<int32_t> all(n);
  for (int32_t i = 0; i < n; ++i) all[i] = i;
  auto o = min_degree(a, all);
  std::copy(o.begin(), o.end(), order);
}

// Exact minimum-degree order of the subgraph induced by verts[0..m), ties to
// the smaller (key[i], verts[i]); key may be NULL (ties to the smaller id).
void oracle_min_degree_keyed(const int32_t* rowptr, const int32_t* col, int32_t n, const int32_t* verts,
                             int32_t m, const uint32_t* key, int32_t* order) {
  Adj a = adj_from_csr(rowptr, col, n);
  std::vector<int32_t> vs(verts, verts + m);
  std::vector<uint32_t> ks;
  if (key) ks.assign(key, key + m);
  auto o = min_degree(a, vs, key ? &ks : nullptr);
  std::copy(o.begin(), o.end(), order);
}

// Keyed minimum-degree orders of several vertex sets at once: set s is
// verts[ptr[s] .. ptr[s+1]), its order is written to the same range of
// `order`; key_of_vertex[v] is the key of vertex v (may be NULL).
void oracle_local_orders_keyed(const int32_t* rowptr, const int32_t* col, int32_t n, const int32_t* ptr,
                               int32_t nsets, const int32_t* verts, const uint32_t* key_of_vertex,
                               int32_t* order) {
  Adj a = adj_from_csr(rowptr, col, n);
  for (int32_t s = 0; s < nsets; ++s) {
    std::vector<int32_t> vs(verts + ptr[s], verts + ptr[s + 1]);
    std::vector<uint32_t> ks;
    for (int32_t v : vs) ks.push_back(key_of_vertex ? key_of_vertex[v] : 0u);
    auto o = min_degree(a, vs, &ks);
    std::copy(o.begin(), o.end(), order + ptr[s]);
  }
}

// The seeded tie-break key of a vertex for the r-th random minimum-degree
// order: the high 32 bits of the seed hash h_r(v) (SplitMix64 at state
// r*gamma + v, as for the patch seeds).
uint32_t oracle_tie_key(uint64_t r, int32_t v) { return (uint32_t)(seed_hash(r, v) >> 32); }

}  // extern "C"

// Algorithm 1 steps 2-4 for given patches: etree (Algorithm 2), local orders
// and their concatenation (Algorithm 3). Outputs as for oracle_order.
static int32_t order_from_patches(const Adj& a, int32_t n, const Patching& P, const oracle_opts* o,
                                  int32_t* label, int32_t* node_of, int32_t* perm, int32_t* iperm,
                                  int32_t* node_begin, int32_t* node_size, int32_t tree_cap, int32_t* depth_out,
                                  int64_t* node_qsum, ND** keep_nd = nullptr) {
  int32_t D = o->nd_level > 0 ? o->nd_level : ceil_log2(P.k);
  int64_t nnodes = ((int64_t)1 << (D + 1)) - 1;
  if (nnodes > tree_cap) return -3;
  ND* ndp = new ND(a, P.label, P.k, D);
  ND& nd = *ndp;
  nd.trace = keep_nd != nullptr;
  std::vector<int32_t> S(P.k), V(n);
  for (int32_t p = 0; p < P.k; ++p) S[p] = p;
  for (int32_t v = 0; v < n; ++v) V[v] = v;
  nd.node(0, 0, S, V);

  std::vector<std::vector<int32_t>> members(nnodes), local(nnodes);
  for (int32_t v = 0; v < n; ++v) members[nd.node_of[v]].push_back(v);
  for (int64_t t = 0; t < nnodes; ++t) local[t] = min_degree(a, members[t]);
  std::vector<int32_t> pv, begin(nnodes, 0);
  if (o->schedule == 0) {
    concat_schedule(0, (int32_t)nnodes, local, pv, begin);
  } else {
    for (int32_t d = D; d >= 0; --d)
      for (int64_t t = ((int64_t)1 << d) - 1; t < ((int64_t)1 << (d + 1)) - 1; ++t) {
        begin[t] = (int32_t)pv.size();
        pv.insert(pv.end(), local[t].begin(), local[t].end());
      }
  }
  for (int32_t i = 0; i < n; ++i) { perm[i] = pv[i]; iperm[pv[i]] = i; }
  std::copy(P.label.begin(), P.label.end(), label);
  std::copy(nd.node_of.begin(), nd.node_of.end(), node_of);
  for (int64_t t = 0; t < nnodes; ++t) { node_begin[t] = begin[t]; node_size[t] = (int32_t)members[t].size(); }
  *depth_out = D;
  if (node_qsum)
    for (int64_t t = 0; t < nnodes; ++t) {
      auto it = nd.qsum_at.find((int32_t)t);
      node_qsum[t] = it == nd.qsum_at.end() ? -1 : it->second;
    }
  if (keep_nd) *keep_nd = ndp; else delete ndp;
  return P.k;
}

extern "C" {

// Algorithm 1: patches -> etree -> perm. Outputs (all caller-allocated):
// label[n] (gmap), node_of[n], perm[n], iperm[n], node_begin/node_size
// [tree_cap] (positions in perm per tree node), *depth_out. Returns k, or a
// negative code: -1 bad options, -3 tree_cap too small.
// node_qsum (nullable, [tree_cap]): for each bisected node, the sum of the
// quotient edge weights w(p,q) over ordered pairs of its patches at the time
// it is bisected; -1 for leaves and unused nodes.
int32_t oracle_order(const int32_t* rowptr, const int32_t* col, int32_t n, const oracle_opts* o,
                     int32_t* label, int32_t* node_of, int32_t* perm, int32_t* iperm,
                     int32_t* node_begin, int32_t* node_size, int32_t tree_cap, int32_t* depth_out,
                     int64_t* node_qsum) {
  if (o->patch_cap < 1 || o->nd_level < 0 || o->lloyd_rounds < 0) return -1;
  Adj a = adj_from_csr(rowptr, col, n);
  Patching P = get_patches(a, o->patch_cap, o->seed, o->lloyd_rounds);
  return order_from_patches(a, n, P, o, label, node_of, perm, iperm, node_begin, node_size, tree_cap, depth_out,
                            node_qsum);
}

// Algorithm 1 with the patches supplied (Section 4, opening: given a patch
// partition, the mesh is not needed): given[v] in [0, k) is the patch of
// vertex v. Groups need not be connected; an empty group has zero weight and
// takes no part in the dissection. patch_cap, seed and lloyd_rounds of `o`
// are not used. Returns k, or -1 (bad options or a label out of range), -3.
int32_t oracle_order_given(const int32_t* rowptr, const int32_t* col, int32_t n, const oracle_opts* o,
                           const int32_t* given, int32_t k, int32_t* label, int32_t* node_of, int32_t* perm,
                           int32_t* iperm, int32_t* node_begin, int32_t* node_size, int32_t tree_cap,
                           int32_t* depth_out, int64_t* node_qsum) {
  if (k < 1 || o->nd_level < 0) return -1;
  for (int32_t v = 0; v < n; ++v)
    if (given[v] < 0 || given[v] >= k) return -1;
  Adj a = adj_from_csr(rowptr, col, n);
  Patching P;
  P.k = k;
  P.label.assign(given, given + n);
  return order_from_patches(a, n, P, o, label, node_of, perm, iperm, node_begin, node_size, tree_cap, depth_out,
                            node_qsum);
}

// Elimination tree and column counts of P (G + I) P^T.
void oracle_symbolic(const int32_t* rowptr, const int32_t* col, int32_t n, const int32_t* perm,
                     int32_t* parent, int32_t* colcount, int64_t* nnzL, int64_t* flops) {
  Adj a = adj_from_csr(rowptr, col, n);
  std::vector<int32_t> p, c;
  symbolic(a, perm, p, c, *nnzL, *flops);
  std::copy(p.begin(), p.end(), parent);
  std::copy(c.begin(), c.end(), colcount);
}

// Section 6.5: expand a vertex ordering and its symbolic results to b degrees
// of freedom per vertex (vertex v owns unknowns b*v .. b*v+b-1). Every
// vertex block is dense, so column b*j+c of L holds the rows b*j+c..b*j+b-1
// of its own block and all b rows of each vertex below j in column j.
void oracle_dof_expand(int32_t n, int32_t b, const int32_t* perm, const int32_t* parent,
                       const int32_t* colcount, int32_t* perm_d, int32_t* parent_d, int32_t* colcount_d) {
  for (int32_t k = 0; k < n; ++k)
    for (int32_t c = 0; c < b; ++c) {
      int64_t i = (int64_t)b * k + c;
      perm_d[i] = b * perm[k] + c;
      if (c < b - 1) parent_d[i] = (int32_t)(i + 1);
      else parent_d[i] = parent[k] < 0 ? -1 : b * parent[k];
      colcount_d[i] = b * colcount[k] - c;
    }
}

}  // extern "C"

extern "C" {

// Patching from explicit seeds (test infrastructure): seeds[0..nseeds) are
// the sources in rank order; then R3 (unreached components), R lloyd_rounds
// and the cap splits follow as in the full method. label_out [n] receives the
// final patch ids, seed_out [n] the seed of every final rank. Returns k.
int32_t oracle_patches_from_seeds(const int32_t* rowptr, const int32_t* col, int32_t n, int32_t nseeds,
                                  const int32_t* seeds, int32_t cap, int32_t lloyd_rounds, int32_t* label_out,
                                  int32_t* seed_out) {
  if (cap < 1 || lloyd_rounds < 0) return -1;
  Adj a = adj_from_csr(rowptr, col, n);
  std::vector<int32_t> s(seeds, seeds + nseeds);
  for (int32_t v : s) if (v < 0 || v >= n) return -1;
  Patching P = patches_from_seeds(a, s, cap, lloyd_rounds, nullptr);
  std::copy(P.label.begin(), P.label.end(), label_out);
  std::copy(P.seed_of.begin(), P.seed_of.end(), seed_out);
  return P.k;
}

// Algorithm 1 with its intermediate stages recorded (test infrastructure).
// given (may be NULL): a supplied patch map with labels in [0, kgiven), as in
// oracle_order_given; the patching rows below are then left untouched.
// Outputs as oracle_order, plus (rows of n ints; entries past the row's
// count are left untouched):
//   seeds0 [n]            seed of every rank after R1 + R3 (*k0_out ranks)
//   lloyd_seeds [R][n]    seed of every rank after each Lloyd round
//   labels [R+1][n]       labels after the first labelling and after each
//                         Lloyd relabel (before the cap splits)
//   side_at, child_at [max_levels][n]: per depth d < D and patch p, the side
//                         p took in the node bisected at depth d and the child
//                         node it moved to (-1 when it has no remaining vertex);
//                         -1 where p took part in no bisection at depth d
// Returns k, or -1 / -3 as oracle_order, or -4 when D > max_levels.
int32_t oracle_order_trace(const int32_t* rowptr, const int32_t* col, int32_t n, const oracle_opts* o,
                           const int32_t* given, int32_t kgiven, int32_t* label, int32_t* node_of, int32_t* perm,
                           int32_t* iperm, int32_t* node_begin, int32_t* node_size, int32_t tree_cap,
                           int32_t* depth_out, int32_t* seeds0, int32_t* k0_out, int32_t* lloyd_seeds,
                           int32_t* labels, int32_t* side_at, int32_t* child_at, int32_t max_levels) {
  if (o->patch_cap < 1 || o->nd_level < 0 || o->lloyd_rounds < 0) return -1;
  Adj a = adj_from_csr(rowptr, col, n);
  PatchTrace tr;
  Patching P;
  if (given) {          // patches supplied: no patching stage to record
    if (kgiven < 1) return -1;
    for (int32_t v = 0; v < n; ++v)
      if (given[v] < 0 || given[v] >= kgiven) return -1;
    P.k = kgiven;
    P.label.assign(given, given + n);
  } else {
    P = get_patches(a, o->patch_cap, o->seed, o->lloyd_rounds, &tr);
  }
  ND* nd = nullptr;
  int32_t k = order_from_patches(a, n, P, o, label, node_of, perm, iperm, node_begin, node_size, tree_cap, depth_out,
                                 nullptr, &nd);
  if (k < 0) return k;
  int32_t D = *depth_out;
  int rc = k;
  if (D > max_levels) rc = -4;
  *k0_out = (int32_t)tr.seeds0.size();
  std::copy(tr.seeds0.begin(), tr.seeds0.end(), seeds0);
  for (size_t r = 0; r < tr.lloyd_seeds.size(); ++r)
    std::copy(tr.lloyd_seeds[r].begin(), tr.lloyd_seeds[r].end(), lloyd_seeds + r * (size_t)n);
  for (size_t r = 0; r < tr.labels.size(); ++r)
    std::copy(tr.labels[r].begin(), tr.labels[r].end(), labels + r * (size_t)n);
  for (int32_t d = 0; d < D && d < max_levels; ++d)
    for (int32_t p = 0; p < k; ++p) {
      bool has = d < (int32_t)nd->side_at.size();
      side_at[(size_t)d * n + p] = has ? nd->side_at[d][p] : -1;
      child_at[(size_t)d * n + p] = has ? nd->child_at[d][p] : -1;
    }
  delete nd;
  return rc;
}

// Quotient graph of a patch map (contract R6, Section 3 definition): node
// weights w[p] = |p|; q_rowptr [k+1], q_col / q_w [cap] list, for every
// patch in increasing neighbour id, the neighbouring patches and the number
// of G-edges between the two. Returns the number of entries (-3 if > cap;
// with q_col NULL only the count).
int64_t oracle_quotient(const int32_t* rowptr, const int32_t* col, int32_t n, const int32_t* label, int32_t k,
                        int32_t* w, int32_t* q_rowptr, int32_t* q_col, int32_t* q_w, int64_t cap) {
  std::vector<std::map<int32_t, int32_t>> q(k);
  std::vector<int32_t> wt(k, 0);
  for (int32_t v = 0; v < n; ++v) {
    wt[label[v]]++;
    for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e)
      if (label[col[e]] != label[v]) q[label[v]][label[col[e]]]++;
  }
  int64_t m = 0;
  for (auto& r : q) m += (int64_t)r.size();
  if (!q_col) return m;
  if (m > cap) return -3;
  int64_t e = 0;
  q_rowptr[0] = 0;
  for (int32_t p = 0; p < k; ++p) {
    w[p] = wt[p];
    for (auto& kv : q[p]) { q_col[e] = kv.first; q_w[e] = kv.second; ++e; }
    q_rowptr[p + 1] = (int32_t)e;
  }
  return m;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Numeric factorisation and solve (Section 6: the permutation and its
// elimination tree drive a sparse Cholesky solver). Textbook up-looking
// sparse Cholesky in FP64 (row k of L solves L[0:k,0:k] l = B[0:k,k] over the
// columns of k's elimination-tree reach; George & Liu 1981, Davis 2006 ch. 4),
// written plainly: a dense accumulator, columns kept as growing lists.
// ---------------------------------------------------------------------------
extern "C" {

// B = P A P^T with A given by its diagonal a_diag[n] and the off-diagonal
// values a_off[] aligned with the symmetric CSR (rowptr, col) of its graph.
// Outputs L in compressed columns, rows ascending (the diagonal first):
// Lp[n+1], Li[nnz], Lx[nnz]; with Li == NULL only Lp is written and the
// entry count returned. Returns nnz(L), -1 if a pivot is not positive, -3 if
// cap is too small.
int64_t oracle_cholesky(const int32_t* rowptr, const int32_t* col, int32_t n, const double* a_diag,
                        const double* a_off, const int32_t* perm, int64_t* Lp, int32_t* Li, double* Lx, int64_t cap) {
  std::vector<int32_t> iperm(n);
  for (int32_t i = 0; i < n; ++i) iperm[perm[i]] = i;
  Adj a = adj_from_csr(rowptr, col, n);
  std::vector<int32_t> parent, cc;
  int64_t nnzL = 0, fl = 0;
  symbolic(a, perm, parent, cc, nnzL, fl);
  if (!Li) {
    Lp[0] = 0;
    for (int32_t j = 0; j < n; ++j) Lp[j + 1] = Lp[j] + cc[j];
    return nnzL;
  }
  if (nnzL > cap) return -3;
  std::vector<std::vector<int32_t>> rows(n);
  std::vector<std::vector<double>> vals(n);
  std::vector<double> x(n, 0.0);
  std::vector<int32_t> mark(n, -1), reach;
  for (int32_t k = 0; k < n; ++k) {
    // scatter column k of B (rows <= k) and find the reach: every column j < k
    // on an etree path from an entry B(i, k), i < k, up to k
    const int32_t v = perm[k];
    double d = a_diag[v];
    reach.clear();
    mark[k] = k;
    for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
      const int32_t i = iperm[col[e]];
      if (i > k) continue;
      x[i] += a_off[e];
      for (int32_t j = i; mark[j] != k; j = parent[j]) {
        mark[j] = k;
        reach.push_back(j);
      }
    }
    std::sort(reach.begin(), reach.end());
    // triangular solve in increasing column order: l_j = x_j / L_jj, then
    // column j's rows below j (and above k) lose L_pj l_j
    for (int32_t j : reach) {
      const double lj = x[j] / vals[j][0];
      x[j] = 0.0;
      for (size_t q = 1; q < rows[j].size(); ++q) x[rows[j][q]] -= vals[j][q] * lj;
      d -= lj * lj;
      rows[j].push_back(k);
      vals[j].push_back(lj);
    }
    if (!(d > 0.0)) return -1;
    rows[k].push_back(k);
    vals[k].push_back(std::sqrt(d));
  }
  int64_t e = 0;
  Lp[0] = 0;
  for (int32_t j = 0; j < n; ++j) {
    for (size_t q = 0; q < rows[j].size(); ++q) { Li[e] = rows[j][q]; Lx[e] = vals[j][q]; ++e; }
    Lp[j + 1] = e;
  }
  return e;
}

// Solves P A P^T y = P b for x = P^T y with the factor of oracle_cholesky:
// forward substitution L z = P b, back substitution L^T y = z, x[perm[i]] = y[i].
void oracle_cholesky_solve(int32_t n, const int32_t* perm, const int64_t* Lp, const int32_t* Li, const double* Lx,
                           const double* b, double* x) {
  std::vector<double> y(n);
  for (int32_t i = 0; i < n; ++i) y[i] = b[perm[i]];
  for (int32_t j = 0; j < n; ++j) {
    y[j] /= Lx[Lp[j]];
    for (int64_t q = Lp[j] + 1; q < Lp[j + 1]; ++q) y[Li[q]] -= Lx[q] * y[j];
  }
  for (int32_t j = n - 1; j >= 0; --j) {
    double s = y[j];
    for (int64_t q = Lp[j] + 1; q < Lp[j + 1]; ++q) s -= Lx[q] * y[Li[q]];
    y[j] = s / Lx[Lp[j]];
  }
  for (int32_t i = 0; i < n; ++i) x[perm[i]] = y[i];
}

}  // extern "C"
