// Host network compiler: from species and reactions to the device tables.
//
// Sec. 4 of the paper builds the incidence matrix of the network and names the
// sparse/dense trade-off of the Jacobian. Here, once per network:
//   1. the stoichiometry nu = products - reactants, as per-species gather lists
//      of signed reaction indices (|nu| copies each), split into segments of at
//      most kSegLen entries so that hub species do not serialise the gather;
//   2. the analytic Jacobian's pattern: J(i,l) != 0 when l is a reactant of a
//      reaction in which species i takes part, plus the diagonal;
//   3. a fill-reducing order: minimum degree on the pattern of J + J^T;
//   4. the symbolic LU of I - cJ in that order (no pivoting; the diagonal of
//      I - cJ is >= 1 for mass-action networks because J(i,i) <= 0), giving
//      per pivot k the rows i > k of L(:,k) and the columns j > k of U(k,:);
//   5. per Jacobian slot, the signed list of reaction-partial indices
//      (2 j + s for d r_j / d x of reactant slot s) that sum into it.
#include <algorithm>
#include <cstdio>
#include <numeric>

#include "internal.h"

namespace cbx {

std::vector<int> minimum_degree_order(const std::vector<uint8_t>& sym, int S) {
  // Explicit elimination graph: eliminate the node of smallest current degree
  // (ties: smallest index), then connect its neighbours pairwise.
  std::vector<std::vector<uint8_t>> adj(S, std::vector<uint8_t>(S, 0));
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j) adj[i][j] = (i != j) && sym[(size_t)i * S + j];
  std::vector<uint8_t> alive(S, 1);
  std::vector<int> deg(S, 0), order;
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j) deg[i] += adj[i][j];
  order.reserve(S);
  std::vector<int> nb;
  for (int step = 0; step < S; ++step) {
    int v = -1;
    for (int i = 0; i < S; ++i)
      if (alive[i] && (v < 0 || deg[i] < deg[v])) v = i;
    order.push_back(v);
    alive[v] = 0;
    nb.clear();
    for (int j = 0; j < S; ++j)
      if (alive[j] && adj[v][j]) nb.push_back(j);
    for (int a : nb) {
      adj[a][v] = adj[v][a] = 0;
      for (int b : nb)
        if (a != b && !adj[a][b]) adj[a][b] = 1;
    }
    for (int a : nb) {
      int d = 0;
      for (int j = 0; j < S; ++j) d += alive[j] && adj[a][j];
      deg[a] = d;
    }
  }
  return order;
}

std::string compile_network(const cbx_species* sp, int S, const cbx_reaction* rx, int R, HostNet* out) {
  char msg[256];
  if (S < 1) return "S must be >= 1";
  if (R < 0) return "R must be >= 0";
  if (!sp) return "species is NULL";
  if (R > 0 && !rx) return "reactions is NULL";
  for (int j = 0; j < R; ++j) {
    const cbx_reaction& r = rx[j];
    if (r.type != CBX_TWO_BODY && r.type != CBX_COSMIC_RAY && r.type != CBX_PHOTO && r.type != CBX_CR_PHOTO) {
      snprintf(msg, sizeof msg, "reaction %d: unknown type %d", j, r.type);
      return msg;
    }
    const bool two = r.type == CBX_TWO_BODY;
    if (r.reac[0] < 0 || r.reac[0] >= S || (two && (r.reac[1] < 0 || r.reac[1] >= S)) ||
        (!two && r.reac[1] != -1)) {
      snprintf(msg, sizeof msg, "reaction %d: reactants (%d, %d) do not fit type %d and S = %d", j,
               r.reac[0], r.reac[1], r.type, S);
      return msg;
    }
    int np = 0;
    for (int p = 0; p < 4; ++p) {
      if (r.prod[p] >= S || r.prod[p] < -1) {
        snprintf(msg, sizeof msg, "reaction %d: product index %d out of range", j, r.prod[p]);
        return msg;
      }
      np += r.prod[p] >= 0;
    }
    if (np == 0) {
      snprintf(msg, sizeof msg, "reaction %d has no product", j);
      return msg;
    }
    if (!(r.alpha == r.alpha) || !(r.beta == r.beta) || !(r.gamma == r.gamma)) {
      snprintf(msg, sizeof msg, "reaction %d has a NaN parameter", j);
      return msg;
    }
  }
  HostNet& n = *out;
  n = HostNet();
  n.S = S;
  n.R = R;
  // net stoichiometry nu[i][j] (user order)
  std::vector<int> nu((size_t)S * R, 0);
  for (int j = 0; j < R; ++j) {
    for (int s = 0; s < 2; ++s)
      if (rx[j].reac[s] >= 0) nu[(size_t)rx[j].reac[s] * R + j] -= 1;
    for (int p = 0; p < 4; ++p)
      if (rx[j].prod[p] >= 0) nu[(size_t)rx[j].prod[p] * R + j] += 1;
  }
  // Jacobian pattern (user order)
  std::vector<uint8_t> pat((size_t)S * S, 0);
  for (int i = 0; i < S; ++i) pat[(size_t)i * S + i] = 1;
  for (int j = 0; j < R; ++j)
    for (int s = 0; s < 2; ++s) {
      const int l = rx[j].reac[s];
      if (l < 0) continue;
      for (int i = 0; i < S; ++i)
        if (nu[(size_t)i * R + j] != 0) pat[(size_t)i * S + l] = 1;
    }
  std::vector<uint8_t> sym(pat);
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j) sym[(size_t)i * S + j] |= pat[(size_t)j * S + i];
  n.perm = minimum_degree_order(sym, S);
  n.iperm.assign(S, 0);
  for (int k = 0; k < S; ++k) n.iperm[n.perm[k]] = k;
  // reactions in internal numbering
  n.rtype.resize(R);
  n.ra.resize(R);
  n.rb.resize(R);
  n.alpha.resize(R);
  n.beta.resize(R);
  n.gamma.resize(R);
  n.rprod.assign((size_t)4 * R, -1);
  for (int j = 0; j < R; ++j) {
    for (int p = 0; p < 4; ++p) n.rprod[4 * j + p] = rx[j].prod[p] >= 0 ? n.iperm[rx[j].prod[p]] : -1;
    n.rtype[j] = rx[j].type;
    n.ra[j] = n.iperm[rx[j].reac[0]];
    n.rb[j] = rx[j].reac[1] >= 0 ? n.iperm[rx[j].reac[1]] : -1;
    n.alpha[j] = rx[j].alpha;
    n.beta[j] = rx[j].beta;
    n.gamma[j] = rx[j].gamma;
  }
  // reactions grouped by rate type (stable within a type)
  for (int t = 0; t < kNumTypes; ++t) {
    n.tptr[t] = (int)n.rj.size();
    for (int j = 0; j < R; ++j)
      if (n.rtype[j] == t) {
        n.rj.push_back(j);
        n.gbeta.push_back(n.beta[j]);
        n.ggamma.push_back(n.gamma[j]);
      }
  }
  n.tptr[kNumTypes] = (int)n.rj.size();
  // right-hand side gather lists, segmented
  n.spec_seg.push_back(0);
  n.seg_ptr.push_back(0);
  for (int k = 0; k < S; ++k) {
    const int i = n.perm[k];
    std::vector<int> ent;
    for (int j = 0; j < R; ++j) {
      const int v = nu[(size_t)i * R + j];
      for (int c = 0; c < std::abs(v); ++c) ent.push_back((j << 1) | (v < 0 ? 1 : 0));
    }
    for (size_t e = 0; e < ent.size(); e += kSegLen) {
      const size_t end = std::min(ent.size(), e + kSegLen);
      n.rhs_ent.insert(n.rhs_ent.end(), ent.begin() + e, ent.begin() + end);
      n.seg_ptr.push_back((int)n.rhs_ent.size());
    }
    n.spec_seg.push_back((int)n.seg_ptr.size() - 1);
  }
  n.nseg = (int)n.seg_ptr.size() - 1;
  // Jacobian slots in internal order, sorted by (row, col), with their terms
  std::vector<uint8_t> ip((size_t)S * S, 0);
  for (int i = 0; i < S; ++i)
    for (int l = 0; l < S; ++l)
      if (pat[(size_t)i * S + l]) ip[(size_t)n.iperm[i] * S + n.iperm[l]] = 1;
  std::vector<int> slot((size_t)S * S, -1);
  n.jrow_ptr.push_back(0);
  for (int i = 0; i < S; ++i) {
    for (int l = 0; l < S; ++l)
      if (ip[(size_t)i * S + l]) {
        slot[(size_t)i * S + l] = (int)n.jrow.size();
        n.jrow.push_back(i);
        n.jcol.push_back(l);
      }
    n.jrow_ptr.push_back((int)n.jrow.size());
  }
  n.nnzJ = (int)n.jrow.size();
  std::vector<std::vector<int>> terms(n.nnzJ);
  for (int j = 0; j < R; ++j)
    for (int s = 0; s < 2; ++s) {
      const int lu = rx[j].reac[s];
      if (lu < 0) continue;
      const int l = n.iperm[lu];
      for (int iu = 0; iu < S; ++iu) {
        const int v = nu[(size_t)iu * R + j];
        if (v == 0) continue;
        const int sl = slot[(size_t)n.iperm[iu] * S + l];
        for (int c = 0; c < std::abs(v); ++c) terms[sl].push_back(((2 * j + s) << 1) | (v < 0 ? 1 : 0));
      }
    }
  // Slots ordered by term count (longest first) and dealt in groups of 32,
  // one group per warp pass; a group's terms are interleaved (term e of lane l
  // at jg_ptr[g] + 32 e + l) so that the warp reads them coalesced and its
  // lanes sum lists of similar length. Padding entries hold term 0 (a valid
  // index that the device does not add).
  std::vector<int> order(n.nnzJ);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return terms[a].size() > terms[b].size(); });
  n.njg = (n.nnzJ + 31) / 32;
  n.jg_ptr.push_back(0);
  for (int g = 0; g < n.njg; ++g) {
    int cnt = 0;
    for (int l = 0; l < 32; ++l) {
      const int idx = g * 32 + l;
      const int s = idx < n.nnzJ ? order[idx] : -1;
      const int len = s >= 0 ? (int)terms[s].size() : 0;
      n.jg_slot.push_back(s);
      n.jg_len.push_back(len);
      cnt = std::max(cnt, len);
    }
    for (int e = 0; e < cnt; ++e)
      for (int l = 0; l < 32; ++l) {
        const int s = n.jg_slot[(size_t)g * 32 + l];
        n.jg_term.push_back(s >= 0 && e < (int)terms[s].size() ? terms[s][e] : 0);
      }
    n.jg_ptr.push_back((int)n.jg_term.size());
  }
  // symbolic LU of the internal pattern
  std::vector<uint8_t> F(ip);
  n.piv_lptr.push_back(0);
  n.piv_uptr.push_back(0);
  double flops = 0;
  for (int k = 0; k < S; ++k) {
    std::vector<int> rows, cols;
    for (int i = k + 1; i < S; ++i)
      if (F[(size_t)i * S + k]) rows.push_back(i);
    for (int j = k + 1; j < S; ++j)
      if (F[(size_t)k * S + j]) cols.push_back(j);
    for (int i : rows)
      for (int j : cols) F[(size_t)i * S + j] = 1;
    n.piv_l.insert(n.piv_l.end(), rows.begin(), rows.end());
    n.piv_u.insert(n.piv_u.end(), cols.begin(), cols.end());
    n.piv_lptr.push_back((int)n.piv_l.size());
    n.piv_uptr.push_back((int)n.piv_u.size());
    flops += (double)rows.size() + 2.0 * rows.size() * cols.size();
  }
  n.nnzLU = 0;
  for (uint8_t v : F) n.nnzLU += v;
  // Pivots k >= kdense are factored as if L(:,k) and U(k,:) were the full
  // ranges k+1..S-1: an entry outside the pattern holds an exact zero, so the
  // extra a_ik u_kj terms are exact zeros and the result is unchanged; in
  // exchange the kernel needs no index lists there. kdense minimises a cost
  // model of the FP64 kernel per pivot: each warp instruction covers 32
  // columns of one row and takes ~20 SM cycles of the FP64 pipe, plus a fixed
  // cost per pivot that is larger with index lists (their loads sit on the
  // critical path) than with index ranges.
  auto pivot_cost = [&](int k, bool dense) {
    const int nl = dense ? S - k - 1 : n.piv_lptr[k + 1] - n.piv_lptr[k];
    const int nu = dense ? S - k - 1 : n.piv_uptr[k + 1] - n.piv_uptr[k];
    return 20.0 * nl * ((nu + 31) / 32) + (dense ? 900.0 : 2500.0);
  };
  {
    double tail = 0.0, best = 0.0;
    for (int k = 0; k < S; ++k) best += pivot_cost(k, false);
    n.kdense = S;
    double head = best;
    for (int k = S - 1; k >= 0; --k) {
      head -= pivot_cost(k, false);
      tail += pivot_cost(k, true);
      if (head + tail < best) {
        best = head + tail;
        n.kdense = k;
      }
    }
  }
  n.head_ints = 2 * (n.kdense + 1) + n.piv_lptr[n.kdense] + n.piv_uptr[n.kdense];
  // Leading 32-wide panels of the FP64 blocked LU (networks whose matrix lives
  // in global memory) whose trailing update is applied from the pivot lists
  // rather than as a dense rank-32 product: a panel counts while the
  // structural work of its update, sum over its pivots of 2 |L(:,k)| |U(k,:)|
  // restricted to the rows and columns after the panel, is below a quarter of
  // the dense update's 2 * 32 * (S - panel end)^2 (a listed update costs a
  // scattered read-modify-write per term, a dense one a register-tiled FMA).
  n.sparse_panels = 0;
  for (int kb = 0; kb + 32 < S; kb += 32) {
    const int ke = kb + 32;
    double work = 0.0;
    for (int k = kb; k < ke; ++k) {
      int nl = 0, nu = 0;
      for (int e = n.piv_lptr[k]; e < n.piv_lptr[k + 1]; ++e) nl += n.piv_l[e] >= ke;
      for (int e = n.piv_uptr[k]; e < n.piv_uptr[k + 1]; ++e) nu += n.piv_u[e] >= ke;
      work += 2.0 * nl * nu;
    }
    if (work >= 0.25 * 2.0 * 32.0 * (double)(S - ke) * (S - ke)) break;
    ++n.sparse_panels;
  }
  n.lu_flops = flops;
  return "";
}

}  // namespace cbx
