// Host side of the C ABI: problem construction, the xBDD compiler and the exact
// verifier.  The device side lives in fsmt_device.cu.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <numeric>
#include <string>
#include <unordered_map>

#include "fsmt_internal.h"

namespace fsmt {

static thread_local std::string g_error;

void set_error(const std::string& msg) { g_error = msg; }

static fsmt_status fail(fsmt_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

// --------------------------------------------------------------- validation --
static fsmt_status check_atom(const Problem& P, int32_t nnz, const int32_t* var, const int64_t* coef, int64_t q0,
                              int32_t rel) {
  if (nnz < 1) return fail(FSMT_EINVAL, "atom with no variables");
  if (rel < FSMT_LE || rel > FSMT_EQ) return fail(FSMT_EINVAL, "unknown atom relation");
  if (q0 >= (int64_t(1) << 53) || q0 <= -(int64_t(1) << 53)) return fail(FSMT_EINVAL, "|q0| must be below 2^53");
  for (int t = 0; t < nnz; ++t) {
    if (var[t] < 0 || var[t] >= P.n_real) return fail(FSMT_EINVAL, "atom variable out of range");
    if (coef[t] == 0) return fail(FSMT_EINVAL, "atom coefficient is zero");
    if (coef[t] >= (1 << 24) || coef[t] <= -(1 << 24)) return fail(FSMT_EINVAL, "|coefficient| must be below 2^24");
    for (int u = 0; u < t; ++u)
      if (var[u] == var[t]) return fail(FSMT_EINVAL, "atom repeats a variable");
  }
  return FSMT_OK;
}

static fsmt_status check_constraint(const Problem& P, int32_t n_atoms_total, int32_t kind, int32_t nlits,
                                    const int32_t* lits, int32_t param) {
  if (nlits < 0) return fail(FSMT_EINVAL, "negative literal count");
  const int64_t n_ids = (int64_t)P.n_bool + n_atoms_total;
  std::vector<int32_t> ids(nlits);
  for (int t = 0; t < nlits; ++t) {
    if (lits[t] < 0 || (lits[t] >> 1) >= n_ids) return fail(FSMT_EINVAL, "literal names an unknown variable or atom");
    ids[t] = lits[t] >> 1;
  }
  std::sort(ids.begin(), ids.end());
  if (std::adjacent_find(ids.begin(), ids.end()) != ids.end())
    return fail(FSMT_EINVAL, "constraint names a variable or atom twice");
  switch (kind) {
    case FSMT_OR:
    case FSMT_XOR:
    case FSMT_NAE:
      break;
    case FSMT_CARD_LE:
      if (param < 0) return fail(FSMT_EINVAL, "CARD_LE needs param >= 0");
      break;
    case FSMT_MUX:
      if (param < 1 || param > 16 || nlits != param + (1 << param))
        return fail(FSMT_EINVAL, "MUX needs nlits == param + 2^param, 1 <= param <= 16");
      break;
    case FSMT_NEQ_OR:
      if (param < 0 || 2 * (int64_t)param > nlits) return fail(FSMT_EINVAL, "NEQ_OR needs 0 <= 2*param <= nlits");
      break;
    default:
      return fail(FSMT_EINVAL, "unknown constraint kind");
  }
  return FSMT_OK;
}

// ---------------------------------------------------- layered xBDD builder --
// The diagram of a constraint is built from a finite-state description of its
// kind: reading the literals in list order, a state summarises what matters of
// the literals read so far, or the value is already decided.  The states
// reachable at each position become decision nodes; building them bottom-up
// with a unique table keyed by (position, hi, lo), and skipping any node whose
// two children coincide, yields the reduced ordered diagram for that order.
static constexpr int kTrue = -1, kFalse = -2;

struct Machine {
  int kind, param, L;
  int init() const { return 0; }
  int step(int t, int s, bool v) const {
    switch (kind) {
      case FSMT_OR:
        return v ? kTrue : 0;
      case FSMT_XOR:
        return s ^ (v ? 1 : 0);
      case FSMT_CARD_LE: {
        int c = s + (v ? 1 : 0);
        return c > param ? kFalse : c;
      }
      case FSMT_NAE: {
        int u = s | (v ? 1 : 2);
        return u == 3 ? kTrue : u;
      }
      case FSMT_MUX:
        if (t < param) return s | ((v ? 1 : 0) << t);
        if (t - param == s) return v ? kTrue : kFalse;
        return s;
      case FSMT_NEQ_OR:
        if (t < 2 * param) {
          if ((t & 1) == 0) return v ? 2 : 1;    // pending pair value + 1
          return ((s - 1) == (v ? 1 : 0)) ? 0 : kTrue;
        }
        return v ? kTrue : 0;
    }
    return kFalse;
  }
  int finish(int s) const {
    switch (kind) {
      case FSMT_XOR:
        return s == 1 ? kTrue : kFalse;
      case FSMT_CARD_LE:
        return kTrue;
      default:
        return kFalse;
    }
  }
};

struct Diagram {
  std::vector<int32_t> level;   // position in the literal list per node, topological order
  std::vector<uint16_t> hi, lo; // child index, V = TRUE, V+1 = FALSE
  uint8_t root = 0;
};

static bool build_diagram(int kind, int param, const int32_t* lits, int L, Diagram& out) {
  Machine M{kind, param, L};
  // forward: reachable undecided states per position
  std::vector<std::vector<int>> states(L + 1);
  states[0].push_back(M.init());
  for (int t = 0; t < L; ++t) {
    std::vector<int>& nxt = states[t + 1];
    for (int s : states[t])
      for (int v = 0; v < 2; ++v) {
        int u = M.step(t, s, v != 0);
        if (u >= 0 && std::find(nxt.begin(), nxt.end(), u) == nxt.end()) nxt.push_back(u);
      }
  }
  // backward: nodes; refs >= 0 are node ids, kTrue / kFalse terminals
  struct Node {
    int level, hi, lo;
  };
  std::vector<Node> nodes;
  std::vector<std::unordered_map<int, int>> ref(L + 1);
  for (int s : states[L]) ref[L][s] = M.finish(s);
  for (int t = L - 1; t >= 0; --t) {
    std::unordered_map<uint64_t, int> unique;
    const bool neg = (lits[t] & 1) != 0;
    for (int s : states[t]) {
      auto child = [&](bool lit_true) {
        int u = M.step(t, s, lit_true);
        return u < 0 ? u : ref[t + 1].at(u);
      };
      int hi = child(!neg), lo = child(neg);  // hi = the variable is TRUE
      int r;
      if (hi == lo) {
        r = hi;
      } else {
        uint64_t key = ((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo;
        auto it = unique.find(key);
        if (it != unique.end()) {
          r = it->second;
        } else {
          r = (int)nodes.size();
          nodes.push_back({t, hi, lo});
          unique.emplace(key, r);
        }
      }
      ref[t][s] = r;
    }
  }
  int root = ref[0].at(M.init());
  // flatten: reachable nodes by level (parents before children)
  std::vector<int> order;
  if (root >= 0) {
    std::vector<char> seen(nodes.size(), 0);
    std::vector<int> stack{root};
    while (!stack.empty()) {
      int u = stack.back();
      stack.pop_back();
      if (u < 0 || seen[u]) continue;
      seen[u] = 1;
      order.push_back(u);
      stack.push_back(nodes[u].hi);
      stack.push_back(nodes[u].lo);
    }
    std::sort(order.begin(), order.end(), [&](int x, int y) {
      return nodes[x].level != nodes[y].level ? nodes[x].level < nodes[y].level : x > y;
    });
  }
  const int V = (int)order.size();
  if (V > kMaxNodesPerDiagram) return false;
  std::unordered_map<int, int> pos;
  for (int i = 0; i < V; ++i) pos[order[i]] = i;
  auto index = [&](int r) { return r == kTrue ? V : (r == kFalse ? V + 1 : pos.at(r)); };
  out.level.resize(V);
  out.hi.resize(V);
  out.lo.resize(V);
  for (int i = 0; i < V; ++i) {
    const Node& n = nodes[order[i]];
    out.level[i] = n.level;
    out.hi[i] = (uint16_t)index(n.hi);
    out.lo[i] = (uint16_t)index(n.lo);
  }
  out.root = (uint8_t)(root >= 0 ? 0 : (root == kTrue ? 0 : 1));
  return true;
}

// ------------------------------------------------------ chunked schedule ----
// Groups the constraints of C_sigma into chunks for the chunked kernel.  The
// constraints are first ordered for locality -- by the smallest and the largest
// id of the variables they touch (Booleans by id, reals after them), coarsely
// then finely -- so that a chunk's constraints share variables.  A chunk then
// takes constraints in that order until it would exceed kChunkMaxCons
// constraints, kChunkMaxNodes nodes or slot_limit distinct variables/atoms
// ("slots").  Every node's label is rewritten to its chunk-local slot, and a
// child that is a terminal to the fixed row max_nodes (TRUE) or max_nodes + 1
// (FALSE).  Returns
// false if a single constraint does not fit a chunk (the warp-per-constraint
// kernel then serves the instance).
// Shared memory of the 1024-thread kernel, two restarts per lane, left for the
// per-slot arrays (512 bytes a slot: probabilities and adjoints) and the staged
// reals (1024 bytes a real: b and dC/db, double-buffered) once the fixed arrays
// and the per-restart objective (up to 4096 restarts) are placed.
constexpr int kChunkWideBytes = 227 * 1024 - (kChunkMaxNodes * 8 + kChunkMaxCons * 16 + kChunkMaxSlots * 16 +
                                              kChunkMaxTerms * 8 + kChunkMaxReals * 4 + kChunkMaxList * 4) - 4096 * 4;
static_assert(kChunkWideBytes >= kChunkMaxSlots * 512 + 8 * 1024, "wide chunk budget");

static bool build_chunks(const Problem& P, Compiled& C, int slot_limit) {
  const int n_obj = C.n_obj;
  C.chunk_con_ptr.assign(1, 0);
  C.chunk_node_ptr.assign(1, 0);
  C.chunk_list_ptr.assign(1, 0);
  C.clist.clear();
  C.chunk_slot_ptr.assign(1, 0);
  C.slot_label.clear();
  C.slot_meta.clear();
  C.chunk_term_ptr.assign(1, 0);
  C.term_var.clear();
  C.chunk_real_ptr.assign(1, 0);
  C.real_id.clear();
  C.term_coef.clear();
  C.ccon.clear();
  C.cnode_slot.clear();
  C.cnode_hilo.clear();
  C.n_chunks = 0;
  C.chunk_slot_cap = 0;
  C.chunk_real_max = 0;
  if (n_obj == 0) return true;
  struct Key {
    int64_t k0, k1, k2, k3;
    int s;
  };
  std::vector<Key> keys(n_obj);
  for (int s = 0; s < n_obj; ++s) {
    int64_t lo = INT64_MAX, hi = -1;
    for (int v = C.con_ptr[s]; v < C.con_ptr[s + 1]; ++v) {
      const int lab = (int)C.node_label[v];
      if (lab < C.n_bool) {
        lo = std::min<int64_t>(lo, lab);
        hi = std::max<int64_t>(hi, lab);
      } else {
        const int i = lab - C.n_bool;
        for (int64_t t = P.atom_ptr[i]; t < P.atom_ptr[i + 1]; ++t) {
          const int64_t id = (int64_t)C.n_bool + P.atom_var[t];
          lo = std::min(lo, id);
          hi = std::max(hi, id);
        }
      }
    }
    if (hi < 0) lo = hi = 0;
    keys[s] = {lo >> 6, hi >> 3, hi, lo, s};
  }
  std::sort(keys.begin(), keys.end(), [](const Key& x, const Key& y) {
    if (x.k0 != y.k0) return x.k0 < y.k0;
    if (x.k1 != y.k1) return x.k1 < y.k1;
    if (x.k2 != y.k2) return x.k2 < y.k2;
    if (x.k3 != y.k3) return x.k3 < y.k3;
    return x.s < y.s;
  });
  // the open chunk's slots and reals: index arrays over all literals / reals (-1 = not
  // in the chunk) and the keys in insertion order, which is also their numbering
  const int n_ids = C.n_bool + C.n_atoms;
  std::vector<int32_t> slot_idx(2 * (size_t)n_ids, -1), real_idx(C.n_real, -1);
  std::vector<int32_t> chunk_slot_keys, chunk_reals;
  int chunk_cons = 0, chunk_nodes = 0, chunk_terms = 0;
  auto atom_terms = [&](int lab) { return lab < C.n_bool ? 0 : C.atom_ptr[lab - C.n_bool + 1] - C.atom_ptr[lab - C.n_bool]; };
  const int tnode = std::max(1, C.max_nodes);  // row of the TRUE terminal in the kernel's message array
  // diagram shapes in literal space: a node testing a negated literal has its
  // children swapped, so diagrams of one kind and size share a shape whatever
  // the polarities; key = V then (hi, lo) per node, terminals V (TRUE), V+1 (FALSE)
  C.shape_ptr.assign(1, 0);
  C.shape_hi.clear();
  C.shape_lo.clear();
  C.shape_grp.clear();
  C.shape_nodes.clear();
  std::unordered_map<std::string, int> shape_of;
  std::vector<int> con_shape;  // per constraint in chunk order
  // per-constraint scratch: polarity of each literal id, and the first node testing it
  std::vector<int8_t> neg_of(n_ids, 0);
  std::vector<int32_t> first_stamp(n_ids, -1), first_node(n_ids, 0);
  std::string key;
  std::vector<uint16_t> shi, slo, sgrp;
  std::vector<uint32_t> seen;
  auto close_chunk = [&]() {
    C.chunk_con_ptr.push_back((int32_t)(C.ccon.size() / 4));
    C.chunk_node_ptr.push_back((int32_t)C.cnode_slot.size());
    C.chunk_list_ptr.push_back((int32_t)C.clist.size());
    // the chunk's atom terms, in slot order
    int tb = 0;
    for (size_t k = C.chunk_slot_ptr.back(); k < C.slot_label.size(); ++k) {
      const int lab = C.slot_label[k] & 0x7fffffff;
      const int tc = atom_terms(lab);
      C.slot_meta.push_back(tc ? ((tb << 16) | tc) : 0);
      for (int j = 0; j < tc; ++j) {
        const int e = C.atom_ptr[lab - C.n_bool] + j;
        C.term_var.push_back(real_idx[C.atom_var[e]]);
        C.term_coef.push_back(C.atom_coef[e]);
      }
      tb += tc;
    }
    C.chunk_term_ptr.push_back((int32_t)C.term_var.size());
    C.chunk_slot_ptr.push_back((int32_t)C.slot_label.size());
    C.chunk_slot_cap = std::max<int32_t>(C.chunk_slot_cap, (int32_t)chunk_slot_keys.size());
    C.chunk_real_max = std::max<int32_t>(C.chunk_real_max, (int32_t)chunk_reals.size());
    C.real_id.insert(C.real_id.end(), chunk_reals.begin(), chunk_reals.end());
    C.chunk_real_ptr.push_back((int32_t)C.real_id.size());
    for (int r : chunk_reals) real_idx[r] = -1;
    chunk_reals.clear();
    ++C.n_chunks;
    for (int k : chunk_slot_keys) slot_idx[k] = -1;
    chunk_slot_keys.clear();
    chunk_cons = chunk_nodes = chunk_terms = 0;
  };
  // small instances: chunks of fewer constraints, so that they still spread over
  // the SMs (148 on B300); large ones fill chunks to kChunkMaxCons
  constexpr int kTargetChunks = 148;
  const int cons_limit = n_obj < kTargetChunks * 16 ? std::max(1, (n_obj + kTargetChunks - 1) / kTargetChunks)
                                                    : kChunkMaxCons;
  // a slot is a literal: (variable or atom, polarity); key 2 * label + negated
  auto slot_key = [](int lab, bool ng) { return 2 * lab + (ng ? 1 : 0); };
  for (const Key& k : keys) {
    const int s = k.s;
    const int b = C.con_ptr[s], V = C.con_ptr[s + 1] - b;
    {
      const int cid = C.con_id[s];
      for (int64_t t = P.con_ptr[cid]; t < P.con_ptr[cid + 1]; ++t)
        neg_of[P.con_lits[t] >> 1] = (int8_t)(P.con_lits[t] & 1);
    }
    // what the constraint would add to the open chunk; a literal or real tested at
    // several nodes is counted at each (conservative)
    int new_slots = 0, new_terms = 0, new_reals = 0;
    for (int v = b; v < b + V; ++v) {
      const int lab = (int)C.node_label[v];
      if (slot_idx[slot_key(lab, neg_of[lab] != 0)] < 0) {
        ++new_slots;
        new_terms += atom_terms(lab);
      }
      if (lab >= C.n_bool)
        for (int e = C.atom_ptr[lab - C.n_bool]; e < C.atom_ptr[lab - C.n_bool + 1]; ++e)
          if (real_idx[C.atom_var[e]] < 0) ++new_reals;
    }
    const int n_slots = (int)chunk_slot_keys.size(), n_reals = (int)chunk_reals.size();
    if (chunk_cons > 0 && (chunk_cons + 1 > cons_limit || chunk_nodes + V > kChunkMaxNodes ||
                           n_slots + new_slots > slot_limit || chunk_terms + new_terms > kChunkMaxTerms ||
                           (int)(C.clist.size() - C.chunk_list_ptr.back()) + V + 3 > kChunkMaxList ||
                           n_reals + new_reals > kChunkMaxReals ||
                           (slot_limit > kChunkSlotsGeneric &&
                            (n_slots + new_slots) * 512 + (n_reals + new_reals) * 1024 > kChunkWideBytes)))
      close_chunk();
    if (V > kChunkMaxNodes) return false;
    C.ccon.push_back(chunk_nodes);
    C.ccon.push_back(V);
    // z: the root flag of a constant diagram, else where its literal list starts
    C.ccon.push_back(V == 0 ? C.con_root[s] : (int32_t)(C.clist.size() - C.chunk_list_ptr.back()));
    C.ccon.push_back(C.con_id[s]);
    key.assign(reinterpret_cast<const char*>(&V), sizeof(V));
    shi.resize(V);
    slo.resize(V);
    sgrp.resize(V);
    for (int v = b; v < b + V; ++v) {
      const int lab = (int)C.node_label[v];
      const bool ng = neg_of[lab] != 0;
      uint16_t h = (uint16_t)(C.node_hilo[v] & 0xffffu), l = (uint16_t)(C.node_hilo[v] >> 16);
      if (ng) std::swap(h, l);
      if (first_stamp[lab] != s) {  // first node of the constraint testing this variable
        first_stamp[lab] = s;
        first_node[lab] = v - b;
      }
      const uint16_t g = (uint16_t)first_node[lab];
      shi[v - b] = h;
      slo[v - b] = l;
      sgrp[v - b] = g;
      key.append(reinterpret_cast<const char*>(&h), 2);
      key.append(reinterpret_cast<const char*>(&l), 2);
      key.append(reinterpret_cast<const char*>(&g), 2);
    }
    auto sh = shape_of.find(key);
    int sid;
    if (sh == shape_of.end()) {
      sid = (int)C.shape_nodes.size();
      shape_of.emplace(key, sid);
      C.shape_hi.insert(C.shape_hi.end(), shi.begin(), shi.end());
      C.shape_lo.insert(C.shape_lo.end(), slo.begin(), slo.end());
      C.shape_grp.insert(C.shape_grp.end(), sgrp.begin(), sgrp.end());
      C.shape_ptr.push_back((int32_t)C.shape_hi.size());
      C.shape_nodes.push_back(0);
    } else {
      sid = sh->second;
    }
    C.shape_nodes[sid] += V;
    con_shape.push_back(sid);
    for (int v = b; v < b + V; ++v) {
      const int lab = (int)C.node_label[v];
      const bool ng = neg_of[lab] != 0;
      const int sk = slot_key(lab, ng);
      int slot = slot_idx[sk];
      if (slot < 0) {
        slot = (int)chunk_slot_keys.size();
        slot_idx[sk] = slot;
        chunk_slot_keys.push_back(sk);
        C.slot_label.push_back(ng ? (int32_t)((uint32_t)lab | 0x80000000u) : lab);
        chunk_terms += atom_terms(lab);
        if (lab >= C.n_bool)
          for (int e = C.atom_ptr[lab - C.n_bool]; e < C.atom_ptr[lab - C.n_bool + 1]; ++e)
            if (real_idx[C.atom_var[e]] < 0) {
              real_idx[C.atom_var[e]] = (int32_t)chunk_reals.size();
              chunk_reals.push_back(C.atom_var[e]);
            }
      }
      C.cnode_slot.push_back((uint32_t)slot * 4u * kSlotStride);  // the slot row's byte offset
      // children in literal space (hi: the literal holds), so a negated literal's
      // node has them swapped; decision nodes keep their index, the TRUE / FALSE
      // terminals become the fixed rows tnode / tnode + 1 after the largest diagram's nodes
      auto child = [&](uint32_t x) {
        return x < (uint32_t)V ? x : (x == (uint32_t)V ? (uint32_t)tnode : (uint32_t)tnode + 1);
      };
      uint32_t h = child(C.node_hilo[v] & 0xffffu), l = child(C.node_hilo[v] >> 16);
      if (ng) std::swap(h, l);
      C.cnode_hilo.push_back(h | (l << 16));
    }
    {  // the constraint's literal list: slot words of its distinct literals, in order of first node
      const size_t n0 = C.cnode_slot.size() - (size_t)V;
      seen.clear();
      for (size_t v = n0; v < C.cnode_slot.size(); ++v)
        if (std::find(seen.begin(), seen.end(), C.cnode_slot[v]) == seen.end()) seen.push_back(C.cnode_slot[v]);
      while (seen.size() % 4) seen.push_back(0);
      C.clist.insert(C.clist.end(), seen.begin(), seen.end());
    }
    if ((int)chunk_slot_keys.size() > slot_limit || chunk_terms > kChunkMaxTerms ||
        (int)chunk_reals.size() > kChunkMaxReals || (int)(C.clist.size() - C.chunk_list_ptr.back()) > kChunkMaxList)
      return false;
    ++chunk_cons;
    chunk_nodes += V;
  }
  if (chunk_cons > 0) close_chunk();
  // the shapes worth a generated routine: the largest node counts, at most
  // kMaxJitShapes, each of at most kMaxJitShapeNodes nodes; their constraints
  // carry the shape's 1-based rank in the high half of their V field
  std::vector<int> order(C.shape_nodes.size());
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int x, int y) { return C.shape_nodes[x] > C.shape_nodes[y]; });
  C.jit_shape.clear();
  std::vector<int> rank(C.shape_nodes.size(), 0);
  for (int x : order) {
    const int V = C.shape_ptr[x + 1] - C.shape_ptr[x];
    if ((int)C.jit_shape.size() >= kMaxJitShapes) break;
    if (V < 1 || V > kMaxJitShapeNodes) continue;
    C.jit_shape.push_back(x);
    rank[x] = (int)C.jit_shape.size();
  }
  C.all_specialized = !con_shape.empty();
  for (size_t k = 0; k < con_shape.size(); ++k) {
    C.ccon[4 * k + 1] |= rank[con_shape[k]] << 16;
    if (rank[con_shape[k]] == 0) C.all_specialized = false;
  }
  return true;
}

// ------------------------------------------------ projection block shapes ---
// A block's shape: its local real count, and per half-space (in constraint order)
// the local reals and integer coefficients; the right-hand sides and the box are
// data.  The most frequent shapes (at most kMaxProjShapes, each of at most
// kMaxProjShapeVars reals, kMaxProjShapeHs half-spaces and kMaxProjShapeNnz
// nonzeros) get run-time generated projection routines (fsmt_jit.cpp); every block
// records its shape's 1-based rank, 0 for the generic path.
static void select_proj_shapes(Compiled& C) {
  const int ncomp = (int)C.comp_var_ptr.size() - 1;
  C.comp_shape.assign(ncomp, 0);
  C.proj_shape_comp.clear();
  std::unordered_map<std::string, int> id_of;
  std::vector<int> first_comp, count;
  std::vector<int> sid(ncomp, -1);
  std::string key;
  for (int c = 0; c < ncomp; ++c) {
    const int nv = C.comp_var_ptr[c + 1] - C.comp_var_ptr[c];
    const int h0 = C.comp_hs_ptr[c], nh = C.comp_hs_ptr[c + 1] - h0;
    const int nz = C.hs_ptr[h0 + nh] - C.hs_ptr[h0];
    if (nv > kMaxProjShapeVars || nh > kMaxProjShapeHs || nz > kMaxProjShapeNnz) continue;
    key.assign(reinterpret_cast<const char*>(&nv), sizeof(nv));
    for (int q = h0; q < h0 + nh; ++q) {
      const int32_t n = C.hs_ptr[q + 1] - C.hs_ptr[q];
      key.append(reinterpret_cast<const char*>(&n), sizeof(n));
      key.push_back((char)C.hs_eq[q]);
      for (int e = C.hs_ptr[q]; e < C.hs_ptr[q + 1]; ++e) {
        key.append(reinterpret_cast<const char*>(&C.hs_lvar[e]), sizeof(int32_t));
        key.append(reinterpret_cast<const char*>(&C.hs_coef[e]), sizeof(float));
      }
    }
    auto it = id_of.find(key);
    if (it == id_of.end()) {
      it = id_of.emplace(key, (int)first_comp.size()).first;
      first_comp.push_back(c);
      count.push_back(0);
    }
    sid[c] = it->second;
    ++count[it->second];
  }
  std::vector<int> order(first_comp.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return count[a] > count[b]; });
  std::vector<int> rank(first_comp.size(), 0);
  for (int x : order) {
    if ((int)C.proj_shape_comp.size() >= kMaxProjShapes) break;
    C.proj_shape_comp.push_back(first_comp[x]);
    rank[x] = (int)C.proj_shape_comp.size();
  }
  for (int c = 0; c < ncomp; ++c)
    if (sid[c] >= 0) C.comp_shape[c] = rank[sid[c]];
}

// ------------------------------------------------- FP32 bound rounding ------
// Largest (upper) or smallest (lower) float f with  f * c <= d  (f * c < d when
// strict), c a nonzero integer below 2^24 in magnitude and d an integer below
// 2^53: a clamp to f then satisfies c*y <= d exactly.  Products are exact in FP64.
static float inward_bound(int64_t c, int64_t d, bool strict) {
  auto ok = [&](float f) {
    double v = (double)f * (double)c;
    return strict ? v < (double)d : v <= (double)d;
  };
  float f = (float)((double)d / (double)c);
  const bool upper = c > 0;  // the feasible side is f <= d/c when c > 0
  if (upper) {
    while (!ok(f)) f = std::nextafter(f, -INFINITY);
    while (ok(std::nextafter(f, INFINITY)) && std::isfinite(std::nextafter(f, INFINITY))) f = std::nextafter(f, INFINITY);
  } else {
    while (!ok(f)) f = std::nextafter(f, INFINITY);
    while (ok(std::nextafter(f, -INFINITY)) && std::isfinite(std::nextafter(f, -INFINITY))) f = std::nextafter(f, -INFINITY);
  }
  return f;
}

static float float_at_most(double x) {  // largest float <= x
  if (std::isinf(x)) return (float)x;
  float f = (float)x;
  while ((double)f > x) f = std::nextafter(f, -INFINITY);
  return f;
}
static float float_at_least(double x) {  // smallest float >= x
  if (std::isinf(x)) return (float)x;
  float f = (float)x;
  while ((double)f < x) f = std::nextafter(f, INFINITY);
  return f;
}

// ------------------------------------------------------------------ compile --
static bool is_unit_atomic(const Problem& P, int c) {
  int64_t s = P.con_ptr[c], e = P.con_ptr[c + 1];
  return P.con_kind[c] == FSMT_OR && e - s == 1 && (P.con_lits[s] >> 1) >= P.n_bool;
}

static fsmt_status compile(const Problem& P, int policy, Compiled& C) {
  C.n_bool = P.n_bool;
  C.n_real = P.n_real;
  C.n_atoms = P.n_atoms();
  C.n_cons = P.n_cons();
  const int n_cons = C.n_cons;
  // an equality atom only as the positive literal of a unit constraint that the
  // projection enforces: Gaussian smoothing gives it probability 0 in C_sigma, and its
  // negation is not a convex set
  for (int c = 0; c < n_cons; ++c)
    for (int64_t t = P.con_ptr[c]; t < P.con_ptr[c + 1]; ++t) {
      const int32_t l = P.con_lits[t];
      if ((l >> 1) < P.n_bool || P.atom_rel[(l >> 1) - P.n_bool] != FSMT_EQ) continue;
      if (!(policy == FSMT_UNIT_PROJECT && is_unit_atomic(P, c) && (l & 1) == 0))
        return fail(FSMT_EINVAL, "constraint " + std::to_string(c) +
                                     ": an equality atom is accepted only as the positive literal of a unit "
                                     "constraint under FSMT_UNIT_PROJECT");
    }
  // schedule: constraints of C_sigma first (original order), then the projected ones
  std::vector<int> sched;
  std::vector<int> projected;
  sched.reserve(n_cons);
  for (int c = 0; c < n_cons; ++c) {
    if (policy == FSMT_UNIT_PROJECT && is_unit_atomic(P, c))
      projected.push_back(c);
    else
      sched.push_back(c);
  }
  C.n_obj = (int32_t)sched.size();
  sched.insert(sched.end(), projected.begin(), projected.end());
  // diagrams
  C.con_ptr.assign(n_cons + 1, 0);
  C.con_id.assign(n_cons, 0);
  C.con_root.assign(n_cons, 0);
  C.node_label.clear();
  C.node_hilo.clear();
  int64_t total = 0;
  // A diagram depends only on the kind, the parameter, the length and which literals
  // are negated; the variables only label its levels.  Each distinct shape is built
  // once and relabelled for every constraint that has it.
  std::unordered_map<std::string, Diagram> shapes;
  std::string key;
  for (int s = 0; s < n_cons; ++s) {
    int c = sched[s];
    int64_t b = P.con_ptr[c], e = P.con_ptr[c + 1];
    const int32_t* lits = P.con_lits.data() + b;
    const int L = (int)(e - b);
    const int32_t head[3] = {P.con_kind[c], P.con_param[c], L};
    key.assign(reinterpret_cast<const char*>(head), sizeof(head));
    for (int t = 0; t < L; t += 8) {
      unsigned char bits = 0;
      for (int u = t; u < std::min(L, t + 8); ++u) bits |= (unsigned char)((lits[u] & 1) << (u - t));
      key.push_back((char)bits);
    }
    auto it = shapes.find(key);
    if (it == shapes.end()) {
      if (shapes.size() >= (1u << 16)) shapes.clear();  // bounded memory on shape-diverse inputs
      Diagram D;
      if (!build_diagram(P.con_kind[c], P.con_param[c], lits, L, D))
        return fail(FSMT_EINVAL, "a diagram exceeds 65,533 decision nodes");
      it = shapes.emplace(key, std::move(D)).first;
    }
    const Diagram& D = it->second;
    const size_t V = D.level.size();
    C.con_id[s] = c;
    C.con_root[s] = D.root;
    C.con_ptr[s] = (int32_t)total;
    total += (int64_t)V;
    if (total > INT32_MAX) return fail(FSMT_EINVAL, "more than 2^31-1 decision nodes");
    for (size_t i = 0; i < V; ++i) {
      C.node_label.push_back((uint32_t)(lits[D.level[i]] >> 1));
      C.node_hilo.push_back((uint32_t)D.hi[i] | ((uint32_t)D.lo[i] << 16));
    }
    if (s < C.n_obj) C.max_nodes = std::max<int32_t>(C.max_nodes, (int32_t)V);
    if (s == C.n_obj - 1) C.n_obj_nodes = total;
  }
  if (C.n_obj == 0) C.n_obj_nodes = 0;
  C.con_ptr[n_cons] = (int32_t)total;
  // atoms, normalised to  q.y - q0 (<= | <) 0
  const int K = C.n_atoms;
  C.atom_ptr.assign(K + 1, 0);
  C.atom_var.assign(P.atom_var.begin(), P.atom_var.end());
  C.atom_coef.resize(P.atom_coef.size());
  C.atom_q0f.resize(K);
  C.atom_q0d.resize(K);
  C.atom_inv_norm.resize(K);
  C.atom_strict.resize(K);
  for (int i = 0; i < K; ++i) {
    const int rel = P.atom_rel[i];
    const bool flip = rel == FSMT_GE || rel == FSMT_GT;
    C.atom_strict[i] = rel == FSMT_EQ ? 2 : (rel == FSMT_LT || rel == FSMT_GT) ? 1 : 0;  // 2: equality
    C.atom_ptr[i + 1] = (int32_t)P.atom_ptr[i + 1];
    double nn = 0.0;
    for (int64_t t = P.atom_ptr[i]; t < P.atom_ptr[i + 1]; ++t) {
      int64_t q = flip ? -P.atom_coef[t] : P.atom_coef[t];
      C.atom_coef[t] = (float)q;
      nn += (double)q * (double)q;
    }
    int64_t q0 = flip ? -P.atom_q0[i] : P.atom_q0[i];
    C.atom_q0f[i] = (float)q0;
    C.atom_q0d[i] = (double)q0;
    C.atom_inv_norm[i] = (float)(1.0 / std::sqrt(nn));
  }
  // chunks of up to kChunkMaxSlots slots when every constraint gets a generated
  // routine (the kernel then holds no per-warp message rows); otherwise, or when
  // run-time compilation is switched off, kChunkSlotsGeneric
  const char* no_jit = std::getenv("FSMT_NO_JIT");
  const bool jit_off = no_jit && no_jit[0] && std::string(no_jit) != "0";
  C.chunked_ok = build_chunks(P, C, jit_off ? kChunkSlotsGeneric : kChunkMaxSlots);
  if (C.chunked_ok && !C.all_specialized && !jit_off) C.chunked_ok = build_chunks(P, C, kChunkSlotsGeneric);
  // projection: box, single-variable unit atoms, half-spaces in constraint order
  C.lo.resize(C.n_real);
  C.hi.resize(C.n_real);
  for (int j = 0; j < C.n_real; ++j) {
    C.lo[j] = float_at_least(P.lo[j]);
    C.hi[j] = float_at_most(P.hi[j]);
  }
  struct HS {
    std::vector<int32_t> var;
    std::vector<int64_t> coef;
    int64_t q0;
    bool eq = false;  // a hyperplane q.y = q0 (an equality unit atom)
  };
  std::vector<HS> hs;
  for (int c : projected) {  // ascending constraint id
    int32_t l = P.con_lits[P.con_ptr[c]];
    int i = (l >> 1) - P.n_bool;
    const int rel = P.atom_rel[i];
    if (rel == FSMT_EQ) {  // positive (checked above): pin one real, or a hyperplane
      const int64_t b = P.atom_ptr[i], e = P.atom_ptr[i + 1];
      if (e - b == 1) {
        const int j = P.atom_var[b];
        const int64_t cj = P.atom_coef[b], q0 = P.atom_q0[i];
        // both sides rounded inward: the box is the value when FP32 holds it, else empty
        const float up = inward_bound(cj, q0, false), dn = inward_bound(-cj, -q0, false);
        if (cj > 0) {
          C.hi[j] = std::min(C.hi[j], up);
          C.lo[j] = std::max(C.lo[j], dn);
        } else {
          C.lo[j] = std::max(C.lo[j], up);
          C.hi[j] = std::min(C.hi[j], dn);
        }
      } else {
        HS h;
        for (int64_t t = b; t < e; ++t) {
          h.var.push_back(P.atom_var[t]);
          h.coef.push_back(P.atom_coef[t]);
        }
        h.q0 = P.atom_q0[i];
        h.eq = true;
        hs.push_back(std::move(h));
      }
      continue;
    }
    const bool flip = rel == FSMT_GE || rel == FSMT_GT;
    bool strict = rel == FSMT_LT || rel == FSMT_GT;
    int64_t sgn = flip ? -1 : 1;
    if (l & 1) {  // negated literal: not(q.y <= q0) -> -q.y < -q0 (and vice versa)
      sgn = -sgn;
      strict = !strict;
    }
    int64_t q0 = sgn * P.atom_q0[i];
    int64_t b = P.atom_ptr[i], e = P.atom_ptr[i + 1];
    if (e - b == 1) {
      int j = P.atom_var[b];
      int64_t cj = sgn * P.atom_coef[b];
      float f = inward_bound(cj, q0, strict);
      if (cj > 0)
        C.hi[j] = std::min(C.hi[j], f);
      else
        C.lo[j] = std::max(C.lo[j], f);
    } else {
      HS h;
      for (int64_t t = b; t < e; ++t) {
        h.var.push_back(P.atom_var[t]);
        h.coef.push_back(sgn * P.atom_coef[t]);
      }
      h.q0 = q0;
      hs.push_back(std::move(h));
    }
  }
  C.empty_boxes = 0;
  for (int j = 0; j < C.n_real; ++j) C.empty_boxes += C.lo[j] > C.hi[j] ? 1 : 0;
  // blocks of reals coupled by half-spaces (union-find)
  std::vector<int> parent(C.n_real);
  std::iota(parent.begin(), parent.end(), 0);
  std::function<int(int)> find = [&](int x) { return parent[x] == x ? x : parent[x] = find(parent[x]); };
  std::vector<char> coupled(C.n_real, 0);
  for (auto& h : hs)
    for (size_t t = 0; t < h.var.size(); ++t) {
      coupled[h.var[t]] = 1;
      int a = find(h.var[0]), b = find(h.var[t]);
      if (a != b) parent[b] = a;
    }
  C.free_var.clear();
  std::unordered_map<int, int> comp_of_root;
  std::vector<std::vector<int>> comp_vars, comp_hs;
  for (int j = 0; j < C.n_real; ++j) {
    if (!coupled[j]) {
      C.free_var.push_back(j);
      continue;
    }
    int r = find(j);
    auto it = comp_of_root.find(r);
    int k;
    if (it == comp_of_root.end()) {
      k = (int)comp_vars.size();
      comp_of_root[r] = k;
      comp_vars.emplace_back();
      comp_hs.emplace_back();
    } else {
      k = it->second;
    }
    comp_vars[k].push_back(j);
  }
  for (size_t x = 0; x < hs.size(); ++x) comp_hs[comp_of_root[find(hs[x].var[0])]].push_back((int)x);
  C.comp_var_ptr.assign(1, 0);
  C.comp_hs_ptr.assign(1, 0);
  C.comp_var.clear();
  C.hs_ptr.assign(1, 0);
  C.hs_lvar.clear();
  C.hs_coef.clear();
  C.hs_q0.clear();
  C.hs_inv_qq.clear();
  C.hs_eq.clear();
  C.comp_max_vars = C.comp_max_hs = C.comp_max_nnz = 0;
  for (size_t k = 0; k < comp_vars.size(); ++k) {
    long nnz = 0;
    for (int x : comp_hs[k]) nnz += (long)hs[x].var.size();
    if (proj_block_words((long)comp_vars[k].size(), (long)comp_hs[k].size(), nnz, 1) > kProjSmemWords)
      return fail(FSMT_EINVAL, "a block of reals coupled by unit atoms (" + std::to_string(comp_vars[k].size()) +
                                   " reals, " + std::to_string(comp_hs[k].size()) + " half-spaces, " +
                                   std::to_string(nnz) + " nonzeros) exceeds the projection kernel's shared memory");
    C.comp_max_vars = std::max<int32_t>(C.comp_max_vars, (int32_t)comp_vars[k].size());
    C.comp_max_hs = std::max<int32_t>(C.comp_max_hs, (int32_t)comp_hs[k].size());
    // local reals numbered in order of first appearance in the block's half-spaces
    // (constraint order), so that blocks of one structure -- a precedence chain of a
    // given length, whatever its reals -- share one shape
    std::unordered_map<int, int> local;
    for (int x : comp_hs[k])
      for (int j : hs[x].var)
        if (local.emplace(j, (int)local.size()).second) C.comp_var.push_back(j);
    C.comp_var_ptr.push_back((int32_t)C.comp_var.size());
    for (int x : comp_hs[k]) {
      const HS& h = hs[x];
      double qq = 0.0;
      for (size_t t = 0; t < h.var.size(); ++t) {
        C.hs_lvar.push_back(local.at(h.var[t]));
        C.hs_coef.push_back((float)h.coef[t]);
        qq += (double)h.coef[t] * (double)h.coef[t];
      }
      C.hs_ptr.push_back((int32_t)C.hs_lvar.size());
      C.hs_q0.push_back((float)h.q0);
      C.hs_inv_qq.push_back((float)(1.0 / qq));
      C.hs_eq.push_back(h.eq ? 1 : 0);
    }
    C.comp_hs_ptr.push_back((int32_t)(C.hs_ptr.size() - 1));
    C.comp_max_nnz = std::max<int32_t>(C.comp_max_nnz, C.hs_ptr.back() - C.hs_ptr[C.comp_hs_ptr[C.comp_hs_ptr.size() - 2]]);
  }
  select_proj_shapes(C);
  return FSMT_OK;
}

// --------------------------------------------------------- exact verifier --
// Arbitrary-precision check of sign(sum_t c_t y_t - q0) for double y: every term
// is an integer times a power of two; terms are aligned at the smallest exponent
// and summed as separate positive and negative magnitudes.
struct Mag {
  std::vector<uint32_t> w;
  void add_shifted(unsigned __int128 v, int shift) {
    int word = shift / 32, bit = shift % 32;
    size_t need = word + 6;
    if (w.size() < need) w.resize(need, 0);
    unsigned __int128 carry = 0;
    // v << bit spans at most 5 words (v < 2^128, bit < 32)
    uint32_t chunk[5];
    unsigned __int128 x = v;
    uint64_t spill = 0;
    for (int i = 0; i < 5; ++i) {
      uint64_t lowpart = (uint64_t)(uint32_t)x;
      uint64_t val = (lowpart << bit) | spill;
      chunk[i] = (uint32_t)val;
      spill = val >> 32;
      x >>= 32;
    }
    for (size_t i = word; i < w.size(); ++i) {
      unsigned __int128 s = (unsigned __int128)w[i] + carry + (i - word < 5 ? chunk[i - word] : 0u);
      w[i] = (uint32_t)s;
      carry = s >> 32;
      if (i - word >= 5 && carry == 0) break;
    }
    if (carry) w.push_back((uint32_t)carry);
  }
};
static int cmp_mag(const Mag& a, const Mag& b) {
  size_t n = std::max(a.w.size(), b.w.size());
  for (size_t i = n; i-- > 0;) {
    uint32_t x = i < a.w.size() ? a.w[i] : 0, y = i < b.w.size() ? b.w[i] : 0;
    if (x != y) return x < y ? -1 : 1;
  }
  return 0;
}

// The exact value of sum_{t != skip} c_t y_t - q0 over atom's terms (skip: a term left
// out, or -1), as positive and negative magnitudes in units of 2^kmin.
static void exact_linear(const Problem& P, int atom, const double* y, int64_t skip, Mag& pos, Mag& neg, int& kmin) {
  struct Term {
    unsigned __int128 mag;
    int exp;
    bool neg;
  };
  std::vector<Term> terms;
  for (int64_t t = P.atom_ptr[atom]; t < P.atom_ptr[atom + 1]; ++t) {
    if (t == skip) continue;
    double v = y[P.atom_var[t]];
    if (v == 0.0) continue;
    int e;
    double f = std::frexp(std::fabs(v), &e);  // |v| = f * 2^e, f in [0.5, 1)
    uint64_t m = (uint64_t)std::ldexp(f, 53);
    int k = e - 53;
    int64_t c = P.atom_coef[t];
    unsigned __int128 mag = (unsigned __int128)m * (uint64_t)(c < 0 ? -c : c);
    terms.push_back({mag, k, (v < 0) != (c < 0)});
  }
  int64_t q0 = P.atom_q0[atom];
  if (q0 != 0) terms.push_back({(unsigned __int128)(uint64_t)(q0 < 0 ? -q0 : q0), 0, q0 > 0});
  kmin = 0;
  if (terms.empty()) return;
  kmin = terms[0].exp;
  for (auto& t : terms) kmin = std::min(kmin, t.exp);
  for (auto& t : terms) (t.neg ? neg : pos).add_shifted(t.mag, t.exp - kmin);
}

static int exact_sign_double(const Problem& P, int atom, const double* y) {
  Mag pos, neg;
  int kmin;
  exact_linear(P, atom, y, -1, pos, neg, kmin);
  return cmp_mag(pos, neg);
}

// (pos - neg) * 2^kmin as a double, negated when `negate`; false when a double cannot
// hold it exactly (more than 53 significant bits, or out of range).
static bool exact_to_double(const Mag& pos, const Mag& neg, int kmin, bool negate, double* out) {
  const int c = cmp_mag(pos, neg);
  if (c == 0) {
    *out = 0.0;
    return true;
  }
  const Mag& big = c > 0 ? pos : neg;
  const Mag& small = c > 0 ? neg : pos;
  std::vector<uint32_t> d(big.w.size(), 0);
  int64_t borrow = 0;
  for (size_t i = 0; i < big.w.size(); ++i) {
    int64_t v = (int64_t)big.w[i] - (i < small.w.size() ? (int64_t)small.w[i] : 0) - borrow;
    borrow = v < 0 ? 1 : 0;
    d[i] = (uint32_t)(v + (borrow << 32));
  }
  int hb = -1, lb = -1;
  for (size_t i = 0; i < d.size(); ++i)
    for (int bit = 0; bit < 32; ++bit)
      if ((d[i] >> bit) & 1u) {
        if (lb < 0) lb = (int)i * 32 + bit;
        hb = (int)i * 32 + bit;
      }
  if (hb - lb + 1 > 53) return false;
  uint64_t m = 0;
  for (int b = hb; b >= lb; --b) m = (m << 1) | ((d[b / 32] >> (b % 32)) & 1u);
  const double v = std::ldexp((double)m, kmin + lb);
  if (!std::isfinite(v) || v == 0.0 || std::ldexp(v, -(kmin + lb)) != (double)m) return false;
  *out = ((c > 0) != negate) ? v : -v;
  return true;
}

static bool atom_true_exact(const Problem& P, int atom, const double* y) {
  int s = exact_sign_double(P, atom, y);  // sign of sum coef y - q0 (original relation)
  switch (P.atom_rel[atom]) {
    case FSMT_LE:
      return s <= 0;
    case FSMT_LT:
      return s < 0;
    case FSMT_GE:
      return s >= 0;
    case FSMT_EQ:
      return s == 0;
    default:
      return s > 0;
  }
}

static bool constraint_value(int kind, int param, const std::vector<char>& t) {
  const int L = (int)t.size();
  int cnt = 0;
  for (char v : t) cnt += v;
  switch (kind) {
    case FSMT_OR:
      return cnt > 0;
    case FSMT_XOR:
      return (cnt & 1) == 1;
    case FSMT_CARD_LE:
      return cnt <= param;
    case FSMT_NAE:
      return cnt > 0 && cnt < L;
    case FSMT_MUX: {
      int idx = 0;
      for (int i = 0; i < param; ++i) idx |= (t[i] ? 1 : 0) << i;
      return t[param + idx] != 0;
    }
    case FSMT_NEQ_OR: {
      for (int i = 0; i < param; ++i)
        if (t[2 * i] != t[2 * i + 1]) return true;
      for (int i = 2 * param; i < L; ++i)
        if (t[i]) return true;
      return false;
    }
  }
  return false;
}

}  // namespace fsmt

// ================================================================== C ABI ==
using namespace fsmt;

int fsmt_fused_limit_ok(const fsmt::Compiled& C);  // fsmt_device.cu

extern "C" {

const char* fsmt_last_error(void) { return g_error.c_str(); }
const char* fsmt_version(void) { return "fsmt-b300 0.1"; }

fsmt_status fsmt_problem_create(int32_t n_bool, int32_t n_real, fsmt_problem** out) {
  if (!out) return fail(FSMT_EINVAL, "out is NULL");
  if (n_bool < 0 || n_real < 0) return fail(FSMT_EINVAL, "negative size");
  try {
    auto* p = new fsmt_problem();
    p->p.n_bool = n_bool;
    p->p.n_real = n_real;
    p->p.lo.assign(n_real, -INFINITY);
    p->p.hi.assign(n_real, INFINITY);
    *out = p;
  } catch (...) {
    return fail(FSMT_ENOMEM, "allocation failed");
  }
  return FSMT_OK;
}

void fsmt_free_problem(fsmt_problem* p) { delete p; }

fsmt_status fsmt_set_real_bounds(fsmt_problem* p, int32_t j, double lo, double hi) {
  if (!p) return fail(FSMT_EINVAL, "problem is NULL");
  if (j < 0 || j >= p->p.n_real) return fail(FSMT_EINVAL, "real index out of range");
  if (std::isnan(lo) || std::isnan(hi) || lo > hi) return fail(FSMT_EINVAL, "invalid bounds");
  p->p.lo[j] = lo;
  p->p.hi[j] = hi;
  return FSMT_OK;
}

fsmt_status fsmt_add_atom(fsmt_problem* p, int32_t nnz, const int32_t* var, const int64_t* coef, int64_t q0,
                          int32_t rel, int32_t* atom_id_out) {
  if (!p || (nnz > 0 && (!var || !coef))) return fail(FSMT_EINVAL, "NULL argument");
  Problem& P = p->p;
  fsmt_status s = check_atom(P, nnz, var, coef, q0, rel);
  if (s != FSMT_OK) return s;
  try {
    P.atom_var.insert(P.atom_var.end(), var, var + nnz);
    P.atom_coef.insert(P.atom_coef.end(), coef, coef + nnz);
    P.atom_ptr.push_back((int64_t)P.atom_var.size());
    P.atom_q0.push_back(q0);
    P.atom_rel.push_back((int8_t)rel);
  } catch (...) {
    return fail(FSMT_ENOMEM, "allocation failed");
  }
  if (atom_id_out) *atom_id_out = P.n_atoms() - 1;
  return FSMT_OK;
}

fsmt_status fsmt_add_atoms(fsmt_problem* p, int32_t count, const int64_t* ptr, const int32_t* var,
                           const int64_t* coef, const int64_t* q0, const int8_t* rel) {
  if (!p || count < 0 || (count > 0 && (!ptr || !q0 || !rel))) return fail(FSMT_EINVAL, "NULL argument");
  Problem& P = p->p;
  for (int32_t t = 0; t < count; ++t) {
    if (ptr[t + 1] < ptr[t]) return fail(FSMT_EINVAL, "atom pointers decrease");
    fsmt_status s = check_atom(P, (int32_t)(ptr[t + 1] - ptr[t]), var + ptr[t], coef + ptr[t], q0[t], rel[t]);
    if (s != FSMT_OK) return s;
  }
  try {
    const int64_t base = (int64_t)P.atom_var.size() - ptr[0];
    P.atom_var.insert(P.atom_var.end(), var + ptr[0], var + ptr[count]);
    P.atom_coef.insert(P.atom_coef.end(), coef + ptr[0], coef + ptr[count]);
    for (int32_t t = 0; t < count; ++t) {
      P.atom_ptr.push_back(base + ptr[t + 1]);
      P.atom_q0.push_back(q0[t]);
      P.atom_rel.push_back(rel[t]);
    }
  } catch (...) {
    return fail(FSMT_ENOMEM, "allocation failed");
  }
  return FSMT_OK;
}

fsmt_status fsmt_add_constraint(fsmt_problem* p, int32_t kind, int32_t nlits, const int32_t* lits, int32_t param) {
  if (!p || (nlits > 0 && !lits)) return fail(FSMT_EINVAL, "NULL argument");
  Problem& P = p->p;
  fsmt_status s = check_constraint(P, P.n_atoms(), kind, nlits, lits, param);
  if (s != FSMT_OK) return s;
  try {
    P.con_kind.push_back((int8_t)kind);
    P.con_param.push_back(param);
    P.con_lits.insert(P.con_lits.end(), lits, lits + nlits);
    P.con_ptr.push_back((int64_t)P.con_lits.size());
  } catch (...) {
    return fail(FSMT_ENOMEM, "allocation failed");
  }
  return FSMT_OK;
}

fsmt_status fsmt_add_constraints(fsmt_problem* p, int32_t count, const int8_t* kind, const int32_t* param,
                                 const int64_t* ptr, const int32_t* lits) {
  if (!p || count < 0 || (count > 0 && (!kind || !param || !ptr))) return fail(FSMT_EINVAL, "NULL argument");
  Problem& P = p->p;
  for (int32_t t = 0; t < count; ++t) {
    if (ptr[t + 1] < ptr[t]) return fail(FSMT_EINVAL, "constraint pointers decrease");
    fsmt_status s = check_constraint(P, P.n_atoms(), kind[t], (int32_t)(ptr[t + 1] - ptr[t]), lits + ptr[t], param[t]);
    if (s != FSMT_OK) return s;
  }
  try {
    const int64_t base = (int64_t)P.con_lits.size() - ptr[0];
    P.con_lits.insert(P.con_lits.end(), lits + ptr[0], lits + ptr[count]);
    for (int32_t t = 0; t < count; ++t) {
      P.con_kind.push_back(kind[t]);
      P.con_param.push_back(param[t]);
      P.con_ptr.push_back(base + ptr[t + 1]);
    }
  } catch (...) {
    return fail(FSMT_ENOMEM, "allocation failed");
  }
  return FSMT_OK;
}

fsmt_status fsmt_repair_equalities(const fsmt_problem* p, double* y, int32_t* ok_out) {
  if (!p || !y || !ok_out) return fail(FSMT_EINVAL, "NULL argument");
  const Problem& P = p->p;
  std::vector<int> eqs;  // the projected equality atoms, in constraint order
  for (int c = 0; c < P.n_cons(); ++c) {
    if (!is_unit_atomic(P, c)) continue;
    const int32_t l = P.con_lits[P.con_ptr[c]];
    const int i = (l >> 1) - P.n_bool;
    if ((l & 1) == 0 && P.atom_rel[i] == FSMT_EQ) eqs.push_back(i);
  }
  std::vector<char> pivot(P.n_real, 0);
  int ok = 1;
  for (int i : eqs) {
    if (exact_sign_double(P, i, y) == 0) continue;
    int64_t tp = -1;  // the last real with coefficient +-1 not yet a pivot
    for (int64_t t = P.atom_ptr[i]; t < P.atom_ptr[i + 1]; ++t)
      if ((P.atom_coef[t] == 1 || P.atom_coef[t] == -1) && !pivot[P.atom_var[t]]) tp = t;
    if (tp < 0) {
      ok = 0;
      continue;
    }
    // y_p = (q0 - sum_{t != p} c_t y_t) / c_p = -(sum_{t != p} c_t y_t - q0) * c_p, c_p = +-1
    Mag pos, neg;
    int kmin;
    exact_linear(P, i, y, tp, pos, neg, kmin);
    double v;
    if (!exact_to_double(pos, neg, kmin, P.atom_coef[tp] > 0, &v)) {
      ok = 0;
      continue;
    }
    y[P.atom_var[tp]] = v;
    pivot[P.atom_var[tp]] = 1;
  }
  for (int i : eqs)
    if (exact_sign_double(P, i, y) != 0) ok = 0;
  *ok_out = ok;
  return FSMT_OK;
}

fsmt_status fsmt_verify_exact(const fsmt_problem* p, const int8_t* x, const double* y, int32_t* sat_out,
                              int32_t* first_violated_out) {
  if (!p || !sat_out || (p->p.n_bool && !x) || (p->p.n_real && !y)) return fail(FSMT_EINVAL, "NULL argument");
  const Problem& P = p->p;
  for (int i = 0; i < P.n_bool; ++i)
    if (x[i] != 1 && x[i] != -1) return fail(FSMT_EINVAL, "x entries must be +-1");
  for (int j = 0; j < P.n_real; ++j)
    if (!std::isfinite(y[j])) return fail(FSMT_EINVAL, "y entries must be finite");
  std::vector<char> t;
  std::vector<signed char> atom_val(P.n_atoms(), -1);
  for (int c = 0; c < P.n_cons(); ++c) {
    t.clear();
    for (int64_t k = P.con_ptr[c]; k < P.con_ptr[c + 1]; ++k) {
      int32_t l = P.con_lits[k];
      int id = l >> 1;
      bool v;
      if (id < P.n_bool) {
        v = x[id] == -1;
      } else {
        int a = id - P.n_bool;
        if (atom_val[a] < 0) atom_val[a] = atom_true_exact(P, a, y) ? 1 : 0;
        v = atom_val[a] != 0;
      }
      t.push_back((v != ((l & 1) != 0)) ? 1 : 0);
    }
    if (!constraint_value(P.con_kind[c], P.con_param[c], t)) {
      *sat_out = 0;
      if (first_violated_out) *first_violated_out = c;
      return FSMT_OK;
    }
  }
  *sat_out = 1;
  if (first_violated_out) *first_violated_out = -1;
  return FSMT_OK;
}

fsmt_status fsmt_compile(const fsmt_problem* p, int32_t unit_policy, fsmt_compiled** out) {
  if (!p || !out) return fail(FSMT_EINVAL, "NULL argument");
  if (unit_policy != FSMT_UNIT_PROJECT && unit_policy != FSMT_UNIT_SOFT) return fail(FSMT_EINVAL, "unknown unit policy");
  fsmt_compiled* c = nullptr;
  try {
    c = new fsmt_compiled();
    fsmt_status s = compile(p->p, unit_policy, c->c);
    if (s != FSMT_OK) {
      delete c;
      return s;
    }
  } catch (const std::bad_alloc&) {
    delete c;
    return fail(FSMT_ENOMEM, "allocation failed");
  } catch (const std::exception& e) {
    delete c;
    return fail(FSMT_EINVAL, e.what());
  }
  *out = c;
  return FSMT_OK;
}

fsmt_status fsmt_compiled_info(const fsmt_compiled* c, fsmt_info* out) {
  if (!c || !out) return fail(FSMT_EINVAL, "NULL argument");
  const Compiled& C = c->c;
  std::memset(out, 0, sizeof(*out));
  out->n_bool = C.n_bool;
  out->n_real = C.n_real;
  out->n_atoms = C.n_atoms;
  out->n_cons = C.n_cons;
  out->n_obj_cons = C.n_obj;
  out->n_nodes = C.con_ptr.empty() ? 0 : C.con_ptr.back();
  out->n_obj_nodes = C.n_obj_nodes;
  out->max_nodes = C.max_nodes;
  out->n_halfspaces = (int32_t)C.hs_q0.size();
  out->n_components = (int32_t)C.comp_var_ptr.size() - 1;
  out->n_free_reals = (int32_t)C.free_var.size();
  out->atom_nnz = (int64_t)C.atom_var.size();
  out->fused_ok = fsmt_fused_limit_ok(C);
  out->n_chunks = C.chunked_ok ? C.n_chunks : 0;
  out->jit_shapes = C.jit_shapes;
  out->proj_shapes = C.proj_shapes;
  out->empty_boxes = C.empty_boxes;
  return FSMT_OK;
}

fsmt_status fsmt_get_diagrams(const fsmt_compiled* c, int32_t* con_ptr, int32_t* con_id, uint8_t* con_root,
                              int32_t* label, uint16_t* hi, uint16_t* lo) {
  if (!c) return fail(FSMT_EINVAL, "NULL argument");
  const Compiled& C = c->c;
  if (con_ptr) std::copy(C.con_ptr.begin(), C.con_ptr.end(), con_ptr);
  if (con_id) std::copy(C.con_id.begin(), C.con_id.end(), con_id);
  if (con_root) std::copy(C.con_root.begin(), C.con_root.end(), con_root);
  for (size_t i = 0; i < C.node_label.size(); ++i) {
    if (label) label[i] = (int32_t)C.node_label[i];
    if (hi) hi[i] = (uint16_t)(C.node_hilo[i] & 0xffff);
    if (lo) lo[i] = (uint16_t)(C.node_hilo[i] >> 16);
  }
  return FSMT_OK;
}

fsmt_status fsmt_get_bounds(const fsmt_compiled* c, float* lo, float* hi) {
  if (!c) return fail(FSMT_EINVAL, "NULL argument");
  if (lo) std::copy(c->c.lo.begin(), c->c.lo.end(), lo);
  if (hi) std::copy(c->c.hi.begin(), c->c.hi.end(), hi);
  return FSMT_OK;
}

}  // extern "C"
