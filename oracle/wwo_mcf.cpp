// CPU oracle, Eq. (2): min-cost flow over the residue dual graph.
// TEST INFRASTRUCTURE ONLY (see wwo.h).
//
// Plain successive shortest paths (Sec. II-C; Ahuja et al. Sec. 9.7): explicit
// arc list with unit capacities, node potentials keeping reduced costs
// non-negative, one binary-heap Dijkstra per unit of supply from an excess node
// to the first deficit node it settles, one augmentation, potential update.
// The ground node G keeps its fixed supply r_G (Sec. II-A).
#include "wwo.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <functional>
#include <queue>
#include <vector>

namespace {

struct Arc {
  int64_t tail, head;
  int64_t cost;
  int flow;        // 0 or 1
  int64_t slot;    // index into the cost planes [4][m][n]
};

struct Graph {
  int64_t m, n, N, G;
  std::vector<Arc> arcs;
  std::vector<std::vector<int64_t>> adj;  // arc ids incident to a node (as tail or head)
};

int64_t node_id(int64_t m, int64_t n, int64_t i, int64_t j) {
  if (i < 0 || j < 0 || i >= m - 1 || j >= n - 1) return (m - 1) * (n - 1);
  return i * (n - 1) + j;
}

void build_graph(const int16_t* costs, int64_t m, int64_t n, Graph& g) {
  g.m = m;
  g.n = n;
  g.G = (m - 1) * (n - 1);
  g.N = g.G + 1;
  g.arcs.clear();
  g.adj.assign(g.N, {});
  const int64_t P = m * n;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j + 1 < n; ++j) {  // h(i,j): above (i-1,j), below (i,j)
      int64_t above = node_id(m, n, i - 1, j), below = node_id(m, n, i, j), k = i * n + j;
      g.arcs.push_back({above, below, costs[0 * P + k], 0, 0 * P + k});
      g.arcs.push_back({below, above, costs[1 * P + k], 0, 1 * P + k});
    }
  for (int64_t i = 0; i + 1 < m; ++i)
    for (int64_t j = 0; j < n; ++j) {  // v(i,j): left (i,j-1), right (i,j)
      int64_t left = node_id(m, n, i, j - 1), right = node_id(m, n, i, j), k = i * n + j;
      g.arcs.push_back({right, left, costs[2 * P + k], 0, 2 * P + k});
      g.arcs.push_back({left, right, costs[3 * P + k], 0, 3 * P + k});
    }
  for (int64_t a = 0; a < (int64_t)g.arcs.size(); ++a) {
    g.adj[g.arcs[a].tail].push_back(a);
    g.adj[g.arcs[a].head].push_back(a);
  }
}

void flows_from_arcs(const Graph& g, int8_t* flows) {
  const int64_t P = g.m * g.n;
  std::fill(flows, flows + 2 * P, 0);
  for (const Arc& a : g.arcs) {
    if (!a.flow) continue;
    int plane = (int)(a.slot / P);
    int64_t k = a.slot % P;
    // planes 0/2 give dk = +1 on their edge, planes 1/3 give dk = -1
    flows[(plane / 2) * P + k] += (plane % 2 == 0) ? 1 : -1;
  }
}

}  // namespace

extern "C" {

int wwo_solve_mcf(const int8_t* res, int32_t ground, const int16_t* costs, int64_t m, int64_t n,
                  int8_t* flows, int64_t* potentials, int64_t* total_cost) {
  Graph g;
  build_graph(costs, m, n, g);
  std::vector<int64_t> excess(g.N);
  for (int64_t p = 0; p < g.G; ++p) excess[p] = res[p];
  excess[g.G] = ground;
  std::vector<int64_t> pot(g.N, 0);
  std::vector<int64_t> dist(g.N, LLONG_MAX);
  std::vector<int64_t> pred_arc(g.N, -1);
  std::vector<char> settled(g.N, 0);
  std::vector<int64_t> touched;
  int status = 0;
  int64_t next_src = 0;
  for (;;) {
    while (next_src < g.N && excess[next_src] <= 0) ++next_src;
    if (next_src >= g.N) break;
    const int64_t s = next_src;
    // Dijkstra on reduced costs c - pot(u) + pot(v) >= 0 from s
    typedef std::pair<int64_t, int64_t> QE;
    std::priority_queue<QE, std::vector<QE>, std::greater<QE>> pq;
    for (int64_t v : touched) {
      dist[v] = LLONG_MAX;
      pred_arc[v] = -1;
      settled[v] = 0;
    }
    touched.clear();
    dist[s] = 0;
    touched.push_back(s);
    pq.push({0, s});
    std::vector<int64_t> order;
    int64_t t = -1;
    while (!pq.empty()) {
      QE top = pq.top();
      pq.pop();
      int64_t u = top.second;
      if (settled[u] || top.first != dist[u]) continue;
      settled[u] = 1;
      order.push_back(u);
      if (excess[u] < 0) {
        t = u;
        break;
      }
      for (int64_t aid : g.adj[u]) {
        const Arc& a = g.arcs[aid];
        int64_t v, c;
        if (a.tail == u && a.flow == 0) {
          v = a.head;
          c = a.cost;
        } else if (a.head == u && a.flow == 1) {
          v = a.tail;
          c = -a.cost;
        } else {
          continue;
        }
        int64_t rc = c - pot[u] + pot[v];
        int64_t nd = dist[u] + rc;
        if (nd < dist[v]) {
          if (dist[v] == LLONG_MAX) touched.push_back(v);
          dist[v] = nd;
          pred_arc[v] = aid;
          pq.push({nd, v});
        }
      }
    }
    if (t < 0) {
      status = -4;
      break;
    }
    const int64_t dt = dist[t];
    for (int64_t v : order) pot[v] += dt - dist[v];  // pot = pi + const; see Sec. 9.7
    // augment one unit along the shortest path s -> t
    int64_t v = t;
    while (v != s) {
      Arc& a = g.arcs[pred_arc[v]];
      if (a.head == v) {
        a.flow = 1;
        v = a.tail;
      } else {
        a.flow = 0;
        v = a.head;
      }
    }
    excess[s] -= 1;
    excess[t] += 1;
  }
  flows_from_arcs(g, flows);
  int64_t cost = 0;
  for (const Arc& a : g.arcs) cost += a.cost * a.flow;
  *total_cost = cost;
  for (int64_t p = 0; p < g.N; ++p) potentials[p] = pot[p];
  return status;
}

int64_t wwo_flow_cost(const int16_t* costs, int64_t m, int64_t n, const int8_t* flows) {
  const int64_t P = m * n;
  int64_t cost = 0;
  for (int plane = 0; plane < 2; ++plane)
    for (int64_t k = 0; k < P; ++k) {
      int dk = flows[plane * P + k];
      if (dk > 1 || dk < -1) return -1;
      if (dk == 1) cost += costs[(2 * plane) * P + k];
      if (dk == -1) cost += costs[(2 * plane + 1) * P + k];
    }
  return cost;
}

int wwo_check_certificate(const int8_t* res, int32_t ground, const int16_t* costs, int64_t m,
                          int64_t n, const int8_t* flows, const int64_t* potentials,
                          int64_t* total_cost, int64_t* bad_index) {
  Graph g;
  build_graph(costs, m, n, g);
  const int64_t P = m * n;
  *bad_index = -1;
  // capacity: |dk| <= 1, and no flow on edges that do not exist
  for (int plane = 0; plane < 2; ++plane)
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j) {
        int64_t k = i * n + j;
        int dk = flows[plane * P + k];
        bool exists = plane == 0 ? (j + 1 < n) : (i + 1 < m);
        if (dk > 1 || dk < -1 || (!exists && dk != 0)) {
          *bad_index = plane * P + k;
          return 1;
        }
      }
  for (Arc& a : g.arcs) {
    int plane = (int)(a.slot / P);
    int64_t k = a.slot % P;
    int dk = flows[(plane / 2) * P + k];
    a.flow = (plane % 2 == 0) ? (dk == 1) : (dk == -1);
  }
  // conservation: out - in = supply at every node, G included
  std::vector<int64_t> net(g.N, 0);
  int64_t cost = 0;
  for (const Arc& a : g.arcs) {
    net[a.tail] += a.flow;
    net[a.head] -= a.flow;
    cost += a.cost * a.flow;
  }
  *total_cost = cost;
  for (int64_t p = 0; p < g.N; ++p) {
    int64_t want = p == g.G ? (int64_t)ground : (int64_t)res[p];
    if (net[p] != want) {
      *bad_index = p;
      return 2;
    }
  }
  // reduced-cost optimality on every residual arc (Ahuja Thm 9.3)
  for (int64_t aid = 0; aid < (int64_t)g.arcs.size(); ++aid) {
    const Arc& a = g.arcs[aid];
    int64_t rc;
    if (a.flow == 0)
      rc = a.cost - potentials[a.tail] + potentials[a.head];
    else
      rc = -a.cost - potentials[a.head] + potentials[a.tail];
    if (rc < 0) {
      *bad_index = aid;
      return 3;
    }
  }
  return 0;
}

int64_t wwo_brute_force(const float* psi, const int16_t* costs, int64_t m, int64_t n) {
  const float kPiF = 3.14159274101257324f;
  auto wc = [&](float d) { return (d > kPiF ? 1 : 0) - (d <= -kPiF ? 1 : 0); };
  const int64_t P = m * n;
  std::vector<int> nh(P, 0), nv(P, 0);
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      int64_t k = i * n + j;
      if (j + 1 < n) nh[k] = wc(psi[k + 1] - psi[k]);
      if (i + 1 < m) nv[k] = wc(psi[k + n] - psi[k]);
    }
  std::vector<int64_t> K(P, 0);
  int64_t best = LLONG_MAX;
  // cost of the edge into pixel k from its left or upper neighbour given dk
  auto edge_cost = [&](int plane, int64_t k, int64_t dk) -> int64_t {
    if (dk == 1) return costs[(2 * plane) * P + k];
    if (dk == -1) return costs[(2 * plane + 1) * P + k];
    return 0;
  };
  std::function<void(int64_t, int64_t)> dfs = [&](int64_t idx, int64_t acc) {
    if (acc >= best) return;
    if (idx == P) {
      best = acc;
      return;
    }
    int64_t i = idx / n, j = idx % n;
    int64_t lo = LLONG_MIN, hi = LLONG_MAX;
    // dk = K_v - K_u + n_e in {-1,0,1}
    if (j > 0) {
      int64_t base = K[idx - 1] - nh[idx - 1];
      lo = std::max(lo, base - 1);
      hi = std::min(hi, base + 1);
    }
    if (i > 0) {
      int64_t base = K[idx - n] - nv[idx - n];
      lo = std::max(lo, base - 1);
      hi = std::min(hi, base + 1);
    }
    for (int64_t kv = lo; kv <= hi; ++kv) {
      int64_t add = 0;
      if (j > 0) add += edge_cost(0, idx - 1, kv - K[idx - 1] + nh[idx - 1]);
      if (i > 0) add += edge_cost(1, idx - n, kv - K[idx - n] + nv[idx - n]);
      K[idx] = kv;
      dfs(idx + 1, acc + add);
    }
  };
  K[0] = 0;
  dfs(1, 0);
  return best;
}

int wwo_feasible(const int8_t* res, int32_t ground, int64_t m, int64_t n) {
  // Dinic max-flow: S -> supply nodes, demand nodes -> T, unit arcs both ways per pixel edge.
  const int64_t G = (m - 1) * (n - 1), N = G + 3, S = G + 1, T = G + 2;
  struct E {
    int64_t to, cap, rev;
  };
  std::vector<std::vector<E>> adj(N);
  auto add = [&](int64_t u, int64_t v, int64_t c) {
    adj[u].push_back({v, c, (int64_t)adj[v].size()});
    adj[v].push_back({u, 0, (int64_t)adj[u].size() - 1});
  };
  int64_t need = 0;
  for (int64_t p = 0; p <= G; ++p) {
    int64_t r = p == G ? ground : res[p];
    if (r > 0) {
      add(S, p, r);
      need += r;
    } else if (r < 0) {
      add(p, T, -r);
    }
  }
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j + 1 < n; ++j) {
      int64_t a = node_id(m, n, i - 1, j), b = node_id(m, n, i, j);
      add(a, b, 1);
      add(b, a, 1);
    }
  for (int64_t i = 0; i + 1 < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      int64_t a = node_id(m, n, i, j - 1), b = node_id(m, n, i, j);
      add(a, b, 1);
      add(b, a, 1);
    }
  int64_t flow = 0;
  std::vector<int64_t> level(N), it(N);
  for (;;) {
    std::fill(level.begin(), level.end(), -1);
    std::queue<int64_t> q;
    level[S] = 0;
    q.push(S);
    while (!q.empty()) {
      int64_t u = q.front();
      q.pop();
      for (const E& e : adj[u])
        if (e.cap > 0 && level[e.to] < 0) {
          level[e.to] = level[u] + 1;
          q.push(e.to);
        }
    }
    if (level[T] < 0) break;
    std::fill(it.begin(), it.end(), 0);
    std::function<int64_t(int64_t, int64_t)> push = [&](int64_t u, int64_t f) -> int64_t {
      if (u == T) return f;
      for (int64_t& k = it[u]; k < (int64_t)adj[u].size(); ++k) {
        E& e = adj[u][k];
        if (e.cap > 0 && level[e.to] == level[u] + 1) {
          int64_t d = push(e.to, std::min(f, e.cap));
          if (d > 0) {
            e.cap -= d;
            adj[e.to][e.rev].cap += d;
            return d;
          }
        }
      }
      return 0;
    };
    for (int64_t f; (f = push(S, LLONG_MAX)) > 0;) flow += f;
  }
  return flow == need ? 1 : 0;
}

}  // extern "C"
