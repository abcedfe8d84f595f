// Partition of a decomposition's subdomains over ranks (one GPU each) for
// distributed training: every rank trains its own subdomains and exchanges
// the interface values of the interfaces it shares with other ranks, as
// Algorithm 1 exchanges them between processes.  The work of a rank is the
// sum of its subdomains' weights (their points); the communication is the
// points of the cut interfaces.  Host code.
//
// Method: recursive bisection.  A set of subdomains for k ranks is split in
// two for floor(k/2) and the rest: side A grows from a seed subdomain by
// repeatedly adding the subdomain most strongly connected to A (interface
// points into A minus interface points to the rest of the set), until A holds
// its share of the weight; the cut is then refined by moving subdomains across
// when that cuts fewer interface points and keeps both sides within 5% of
// their shares.  Four growths are tried (seeds at the lowest- and the
// highest-numbered subdomain; ties between equal gains to the lower number or
// to the nearer subdomain in hops from the seed, which grows compact blocks)
// and the smallest cut is kept; then each side is split in turn.
// Deterministic.
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "xpinn.h"

namespace xp {
void set_last_error(const char* msg);
}

namespace {

struct Graph {
  const double* w;
  std::vector<std::vector<std::pair<int, double>>> adj;
};

// One bisection of `nodes` (ascending) into A (side 1, for k1 of the k parts)
// and B (side 2): growth from `seed`, ties between equal gains to the lower
// hop distance from the seed when by_dist (compact blocks), else to the lower
// number; then refinement.  Returns the cut weight; side[] holds the result.
double grow_and_refine(const Graph& g, const std::vector<int>& nodes, int k1, int k2, int seed, bool by_dist,
                       std::vector<int>& side) {
  double W = 0;
  for (int q : nodes) W += g.w[q];
  const double target = W * k1 / (k1 + k2);
  for (int q : nodes) side[q] = 2;
  // hop distance from the seed inside the set (breadth first)
  std::vector<int> dist(g.adj.size(), 1 << 30);
  {
    std::vector<int> fr{seed};
    dist[seed] = 0;
    for (size_t h = 0; h < fr.size(); ++h)
      for (const auto& nb : g.adj[fr[h]])
        if (side[nb.first] == 2 && dist[nb.first] > dist[fr[h]] + 1) {
          dist[nb.first] = dist[fr[h]] + 1;
          fr.push_back(nb.first);
        }
  }
  double wA = 0;
  int nA = 0;
  const int nmax_A = (int)nodes.size() - k2;   // B keeps at least k2 subdomains
  while (nA < nmax_A) {
    int best = -1;
    double best_gain = -1e300;
    if (nA == 0) {
      best = seed;
    } else {
      for (int q : nodes) {
        if (side[q] != 2) continue;
        double in = 0, out = 0;
        bool touches = false;
        for (const auto& nb : g.adj[q]) {
          if (side[nb.first] == 1) {
            in += nb.second;
            touches = true;
          } else if (side[nb.first] == 2) {
            out += nb.second;
          }
        }
        if (!touches) continue;
        const double gain = in - out;
        if (gain > best_gain || (by_dist && gain == best_gain && dist[q] < dist[best])) {
          best_gain = gain;
          best = q;
        }
      }
    }
    if (best < 0)   // A's region is closed: continue from the lowest-numbered rest
      for (int q : nodes)
        if (side[q] == 2) {
          best = q;
          break;
        }
    if (best < 0) break;
    if (nA >= k1 && wA + g.w[best] - target > target - wA) break;   // would overshoot more than it gains
    side[best] = 1;
    wA += g.w[best];
    ++nA;
    if (wA >= target && nA >= k1) break;
  }
  // refinement of the cut, both sides within 5% of their shares
  const double loA = 0.95 * target, hiA = 1.05 * target, W_B = W - target;
  for (int pass = 0; pass < 20; ++pass) {
    bool moved = false;
    for (int q : nodes) {
      double same = 0, other = 0;
      for (const auto& nb : g.adj[q]) {
        if (side[nb.first] == 0) continue;
        (side[nb.first] == side[q] ? same : other) += nb.second;
      }
      if (other <= same) continue;
      if (side[q] == 1) {
        if (nA <= k1 || wA - g.w[q] < loA || (W - wA) + g.w[q] > 1.05 * W_B + 1e-12) continue;
        side[q] = 2;
        wA -= g.w[q];
        --nA;
      } else {
        const int nB = (int)nodes.size() - nA;
        if (nB <= k2 || wA + g.w[q] > hiA || (W - wA) - g.w[q] < 0.95 * W_B - 1e-12) continue;
        side[q] = 1;
        wA += g.w[q];
        ++nA;
      }
      moved = true;
    }
    if (!moved) break;
  }
  double cut = 0;
  for (int q : nodes)
    if (side[q] == 1)
      for (const auto& nb : g.adj[q])
        if (side[nb.first] == 2) cut += nb.second;
  return cut;
}

// Splits `nodes` (ascending) for k parts, numbering them from part0: the
// bisection with the smallest cut among growths from the lowest- and the
// highest-numbered subdomain, ties by number or by distance.
void bisect(const Graph& g, const std::vector<int>& nodes, int k, int part0, std::vector<int>& part,
            std::vector<int>& side) {
  if (k == 1 || nodes.size() <= 1) {
    for (int q : nodes) part[q] = part0;
    return;
  }
  const int k1 = k / 2, k2 = k - k1;
  std::vector<int> best_side;
  double best_cut = 1e300;
  for (int seed : {nodes.front(), nodes.back()})
    for (bool by_dist : {false, true}) {
      const double cut = grow_and_refine(g, nodes, k1, k2, seed, by_dist, side);
      if (cut < best_cut) {
        best_cut = cut;
        best_side.assign(nodes.size(), 0);
        for (size_t i = 0; i < nodes.size(); ++i) best_side[i] = side[nodes[i]];
      }
      for (int q : nodes) side[q] = 0;
    }
  std::vector<int> A, B;
  for (size_t i = 0; i < nodes.size(); ++i) (best_side[i] == 1 ? A : B).push_back(nodes[i]);
  bisect(g, A, k1, part0, part, side);
  bisect(g, B, k2, part0 + k1, part, side);
}

}  // namespace

extern "C" int xpinn_partition(int32_t n_sub, const double* weight, int32_t n_edge, const int32_t* eq,
                               const int32_t* eqp, const double* edge_w, int32_t n_parts, int32_t* part) {
  if (n_sub < 1 || !weight || n_edge < 0 || (n_edge && (!eq || !eqp || !edge_w)) || n_parts < 1 ||
      n_parts > n_sub || !part) {
    xp::set_last_error("xpinn_partition: bad arguments");
    return XPINN_ERR_INVALID;
  }
  for (int e = 0; e < n_edge; ++e)
    if (eq[e] < 0 || eq[e] >= n_sub || eqp[e] < 0 || eqp[e] >= n_sub || !(edge_w[e] >= 0)) {
      xp::set_last_error("xpinn_partition: bad edge");
      return XPINN_ERR_INVALID;
    }
  for (int q = 0; q < n_sub; ++q)
    if (!(weight[q] >= 0)) {
      xp::set_last_error("xpinn_partition: bad weight");
      return XPINN_ERR_INVALID;
    }
  Graph g;
  g.w = weight;
  g.adj.resize(n_sub);
  for (int e = 0; e < n_edge; ++e) {
    if (eq[e] == eqp[e]) continue;
    g.adj[eq[e]].emplace_back(eqp[e], edge_w[e]);
    g.adj[eqp[e]].emplace_back(eq[e], edge_w[e]);
  }
  std::vector<int> nodes(n_sub), P(n_sub, 0), side(n_sub, 0);
  for (int q = 0; q < n_sub; ++q) nodes[q] = q;
  bisect(g, nodes, n_parts, 0, P, side);
  for (int q = 0; q < n_sub; ++q) part[q] = P[q];
  xp::set_last_error("");
  return XPINN_OK;
}
