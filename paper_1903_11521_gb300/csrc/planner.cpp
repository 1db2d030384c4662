// Planner of Einstein-notation tensor operations (Sec. 4): parsing (Sec. 4.1),
// equivalent sparsity patterns (Sec. 4.2, Eq. compeqspp), strength reduction with the
// sparse cost (Sec. 4.3) and optimal index permutations of the temporaries by dynamic
// programming with the Loop-over-GEMM cost (Sec. 4.5, Eqs. permopt, permcost, subproblem).
#include "planner.h"

#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstdlib>
#include <functional>
#include <map>
#include <numeric>
#include <set>

#include "common.h"

namespace yt {
namespace plan {

namespace {

constexpr size_t kMaxPatternSize = size_t(1) << 24;

std::vector<size_t> strides_of(const std::vector<int>& dims) {
  std::vector<size_t> s(dims.size());
  size_t acc = 1;
  for (size_t i = 0; i < dims.size(); ++i) {
    s[i] = acc;
    acc *= (size_t)dims[i];
  }
  return s;
}

size_t volume(const std::vector<int>& dims) {
  size_t v = 1;
  for (int d : dims) {
    v *= (size_t)d;
    if (v > kMaxPatternSize) throw Error(YT_ERR_UNSUPPORTED, "intermediate tensor too large for the planner");
  }
  return v;
}

// Calls f(multi-index) for every point of a column-major space, first index fastest.
template <typename F>
void for_each_point(const std::vector<int>& dims, F f) {
  const size_t n = volume(dims);
  std::vector<int> i(dims.size(), 0);
  for (size_t lin = 0; lin < n; ++lin) {
    f(i, lin);
    for (size_t d = 0; d < dims.size(); ++d) {
      if (++i[d] < dims[d]) break;
      i[d] = 0;
    }
  }
}

size_t product_volume(const BPat& a, const BPat& b) {
  size_t v = 1;
  for (int d : a.dims) v *= (size_t)d;
  for (size_t i = 0; i < b.idx.size(); ++i)
    if (a.idx.find(b.idx[i]) == std::string::npos) {
      v *= (size_t)b.dims[i];
      if (v > kMaxPatternSize) return v;
    }
  return v;
}

BPat from_tensor(const TensorInfo& t, const std::string& idx) {
  BPat p;
  p.idx = idx;
  p.dims = t.shape;
  p.bits = t.pattern;
  return p;
}

}  // namespace

int64_t BPat::nnz() const {
  int64_t n = 0;
  for (uint8_t b : bits) n += b != 0;
  return n;
}

BPat product(const BPat& a, const BPat& b) {
  BPat r;
  r.idx = a.idx;
  r.dims = a.dims;
  for (size_t i = 0; i < b.idx.size(); ++i)
    if (a.idx.find(b.idx[i]) == std::string::npos) {
      r.idx.push_back(b.idx[i]);
      r.dims.push_back(b.dims[i]);
    }
  r.bits.assign(volume(r.dims), 0);
  const auto sa = strides_of(a.dims), sb = strides_of(b.dims);
  std::vector<size_t> ma(r.idx.size(), 0), mb(r.idx.size(), 0);
  for (size_t d = 0; d < r.idx.size(); ++d) {
    const auto pa = a.idx.find(r.idx[d]), pb = b.idx.find(r.idx[d]);
    if (pa != std::string::npos) ma[d] = sa[pa];
    if (pb != std::string::npos) mb[d] = sb[pb];
  }
  for_each_point(r.dims, [&](const std::vector<int>& i, size_t lin) {
    size_t oa = 0, ob = 0;
    for (size_t d = 0; d < i.size(); ++d) {
      oa += i[d] * ma[d];
      ob += i[d] * mb[d];
    }
    r.bits[lin] = a.bits[oa] && b.bits[ob];
  });
  return r;
}

BPat sum_out(const BPat& v, const std::string& keep) {
  BPat r;
  for (size_t d = 0; d < v.idx.size(); ++d)
    if (keep.find(v.idx[d]) != std::string::npos) {
      r.idx.push_back(v.idx[d]);
      r.dims.push_back(v.dims[d]);
    }
  if (r.idx.size() == v.idx.size()) return v;
  r.bits.assign(volume(r.dims), 0);
  const auto sr = strides_of(r.dims);
  std::vector<size_t> m(v.idx.size(), 0);
  for (size_t d = 0; d < v.idx.size(); ++d) {
    const auto p = r.idx.find(v.idx[d]);
    if (p != std::string::npos) m[d] = sr[p];
  }
  for_each_point(v.dims, [&](const std::vector<int>& i, size_t lin) {
    if (!v.bits[lin]) return;
    size_t o = 0;
    for (size_t d = 0; d < i.size(); ++d) o += i[d] * m[d];
    r.bits[o] = 1;
  });
  return r;
}

BPat permute(const BPat& v, const std::string& order) {
  if (order == v.idx) return v;
  BPat r;
  r.idx = order;
  for (char c : order) {
    const auto p = v.idx.find(c);
    if (p == std::string::npos) throw Error(YT_ERR_INVALID, "permute: index sets differ");
    r.dims.push_back(v.dims[p]);
  }
  r.bits.assign(v.bits.size(), 0);
  const auto sv = strides_of(v.dims);
  std::vector<size_t> m(order.size());
  for (size_t d = 0; d < order.size(); ++d) m[d] = sv[v.idx.find(order[d])];
  for_each_point(r.dims, [&](const std::vector<int>& i, size_t lin) {
    size_t o = 0;
    for (size_t d = 0; d < i.size(); ++d) o += i[d] * m[d];
    r.bits[lin] = v.bits[o];
  });
  return r;
}

// ------------------------------------------------------------------------- parsing
namespace {

struct Lexer {
  const std::string& s;
  size_t p = 0;
  explicit Lexer(const std::string& str) : s(str) {}
  void ws() {
    while (p < s.size() && std::isspace((unsigned char)s[p])) ++p;
  }
  bool eat(const char* tok) {
    ws();
    const size_t n = std::char_traits<char>::length(tok);
    if (s.compare(p, n, tok) == 0) {
      p += n;
      return true;
    }
    return false;
  }
  bool at_end() {
    ws();
    return p >= s.size();
  }
  bool peek_number() {
    ws();
    return p < s.size() && (std::isdigit((unsigned char)s[p]) || s[p] == '.' || s[p] == '-' || s[p] == '+');
  }
  double number() {
    ws();
    const char* begin = s.c_str() + p;
    char* end = nullptr;
    const double v = std::strtod(begin, &end);
    if (end == begin) throw Error(YT_ERR_PARSE, "expected a number at position " + std::to_string(p));
    p += (size_t)(end - begin);
    return v;
  }
  std::string name() {
    ws();
    const size_t b = p;
    while (p < s.size() && (std::isalnum((unsigned char)s[p]) || s[p] == '_')) ++p;
    if (b == p) throw Error(YT_ERR_PARSE, "expected a tensor name at position " + std::to_string(b));
    return s.substr(b, p - b);
  }
  std::string indices() {
    if (!eat("[")) throw Error(YT_ERR_PARSE, "expected '[' at position " + std::to_string(p));
    ws();
    const size_t b = p;
    while (p < s.size() && std::isalpha((unsigned char)s[p])) ++p;
    std::string idx = s.substr(b, p - b);
    if (!eat("]")) throw Error(YT_ERR_PARSE, "expected ']' (indices are letters a-z, A-Z) at position " + std::to_string(p));
    return idx;
  }
};

int find_tensor(const std::vector<TensorInfo>& t, const std::string& name) {
  for (size_t i = 0; i < t.size(); ++i)
    if (t[i].name == name) return (int)i;
  throw Error(YT_ERR_PARSE, "unknown tensor '" + name + "'");
}

void check_factor(const TensorInfo& t, const std::string& idx) {
  if ((int)idx.size() != (int)t.shape.size())
    throw Error(YT_ERR_SHAPE, "index string of " + t.name + " must have one letter per dimension");
  std::set<char> seen(idx.begin(), idx.end());
  if (seen.size() != idx.size())
    throw Error(YT_ERR_PARSE, "repeated index inside " + t.name + " (a trace is not an Einstein product)");
}

}  // namespace

Expression parse(const std::string& text, const std::vector<TensorInfo>& tensors) {
  Lexer lx(text);
  Expression e;
  e.lhs = find_tensor(tensors, lx.name());
  e.lhs_idx = lx.indices();
  check_factor(tensors[e.lhs], e.lhs_idx);
  if (tensors[e.lhs].global) throw Error(YT_ERR_INVALID, "the result tensor must be per-element");
  if (lx.eat("+=")) e.accumulate = true;
  else if (!lx.eat("=")) throw Error(YT_ERR_PARSE, "expected '=' or '+='");
  for (;;) {
    Term t;
    if (lx.peek_number()) {
      t.scalar = lx.number();
      if (!lx.eat("*")) throw Error(YT_ERR_PARSE, "expected '*' after a scalar");
    }
    for (;;) {
      Factor f;
      f.tensor = find_tensor(tensors, lx.name());
      f.idx = lx.indices();
      check_factor(tensors[f.tensor], f.idx);
      if (f.tensor == e.lhs) throw Error(YT_ERR_UNSUPPORTED, "the result tensor may not appear on the right-hand side");
      t.factors.push_back(f);
      if (!lx.eat("*")) break;
    }
    e.terms.push_back(t);
    if (lx.at_end()) break;
    if (!lx.eat("+")) throw Error(YT_ERR_PARSE, "expected '+' or end of expression at position " + std::to_string(lx.p));
  }
  // sizes consistent per term, result indices covered
  for (const Term& t : e.terms) {
    std::map<char, int> size;
    auto bind = [&](const std::string& idx, const TensorInfo& ti) {
      for (size_t d = 0; d < idx.size(); ++d) {
        auto it = size.find(idx[d]);
        if (it == size.end()) size[idx[d]] = ti.shape[d];
        else if (it->second != ti.shape[d])
          throw Error(YT_ERR_SHAPE, std::string("inconsistent size of index '") + idx[d] + "'");
      }
    };
    bind(e.lhs_idx, tensors[e.lhs]);
    std::set<char> rhs;
    for (const Factor& f : t.factors) {
      bind(f.idx, tensors[f.tensor]);
      rhs.insert(f.idx.begin(), f.idx.end());
    }
    for (char c : e.lhs_idx)
      if (!rhs.count(c)) throw Error(YT_ERR_SHAPE, std::string("result index '") + c + "' does not occur in a term");
    if (t.factors.size() > 12) throw Error(YT_ERR_UNSUPPORTED, "at most 12 factors per term");
  }
  return e;
}

// -------------------------------------------------------------------------- EQSPP
std::vector<BPat> eqspp(const Term& term, const std::vector<TensorInfo>& tensors) {
  const size_t n = term.factors.size();
  std::vector<BPat> pats(n), out(n);
  for (size_t k = 0; k < n; ++k) pats[k] = from_tensor(tensors[term.factors[k].tensor], term.factors[k].idx);
  for (size_t k = 0; k < n; ++k) {
    // contraction of all other patterns onto the indices of factor k (OR over the rest)
    std::vector<BPat> rest;
    for (size_t m = 0; m < n; ++m)
      if (m != k) rest.push_back(pats[m]);
    auto needed = [&](size_t skip_a, size_t skip_b) {
      std::string keep = pats[k].idx;
      for (size_t m = 0; m < rest.size(); ++m)
        if (m != skip_a && m != skip_b) keep += rest[m].idx;
      return keep;
    };
    for (size_t m = 0; m < rest.size(); ++m) rest[m] = sum_out(rest[m], needed(m, m));
    while (rest.size() > 1) {
      size_t ba = 0, bb = 1;
      size_t best = SIZE_MAX;
      for (size_t a = 0; a < rest.size(); ++a)
        for (size_t b = a + 1; b < rest.size(); ++b) {
          std::string u = rest[a].idx;
          size_t vol = rest[a].size();
          for (size_t d = 0; d < rest[b].idx.size(); ++d)
            if (u.find(rest[b].idx[d]) == std::string::npos) {
              u.push_back(rest[b].idx[d]);
              vol *= (size_t)rest[b].dims[d];
            }
          if (vol < best) { best = vol; ba = a; bb = b; }
        }
      BPat pr = sum_out(product(rest[ba], rest[bb]), needed(ba, bb));
      rest.erase(rest.begin() + bb);
      rest[ba] = pr;
    }
    BPat q = pats[k];
    if (!rest.empty()) q = product(pats[k], rest[0]);      // AND with Theta^k itself
    out[k] = sum_out(q, pats[k].idx);
    out[k] = permute(out[k], pats[k].idx);
  }
  return out;
}

// ----------------------------------------------------------------------- LoG cost
namespace {
// All runs of consecutive characters of `src` whose characters are all in `set` and that
// also occur consecutively and in the same order in `other`.  A GEMM block may be empty
// only when its index class is empty: every class of free / contracted indices takes
// part in the GEMM with at least one index.
std::vector<std::string> runs(const std::string& src, const std::string& set, const std::string& other) {
  std::vector<std::string> r;
  if (set.empty()) r.push_back(std::string());
  for (size_t p = 0; p < src.size(); ++p) {
    for (size_t len = 1; p + len <= src.size(); ++len) {
      const char c = src[p + len - 1];
      if (set.find(c) == std::string::npos) break;
      const std::string g = src.substr(p, len);
      const auto q = other.find(g);
      if (q != std::string::npos) r.push_back(g);
    }
  }
  return r;
}
long pos(const std::string& s, const std::string& g) {
  return g.empty() ? -1 : (long)s.find(g[0]);
}
}  // namespace

LogCost min_log(const std::string& c, const std::string& a, const std::string& b) {
  bool found = false;
  LogCost best;
  for (int role = 0; role < 2; ++role) {
    const std::string& L = role == 0 ? a : b;
    const std::string& R = role == 0 ? b : a;
    std::string mset, nset, kset;
    for (char x : L) {
      const bool inR = R.find(x) != std::string::npos, inC = c.find(x) != std::string::npos;
      if (inC && !inR) mset.push_back(x);
      if (inR && !inC) kset.push_back(x);
    }
    for (char x : R)
      if (c.find(x) != std::string::npos && L.find(x) == std::string::npos) nset.push_back(x);
    const auto Ms = runs(L, mset, c), Ns = runs(R, nset, c), Ks = runs(L, kset, R);
    for (const auto& M : Ms)
      for (const auto& Nn : Ns)
        for (const auto& K : Ks) {
          if (!M.empty() && !Nn.empty() && pos(c, M) > pos(c, Nn)) continue;
          LogCost cost;
          // C: leading block M (or N if no M)
          const std::string& c_first = !M.empty() ? M : Nn;
          if (!c_first.empty() && pos(c, c_first) != 0) cost.s += 1;
          // L: blocks M and K
          long lm = pos(L, M), lk = pos(L, K);
          long lfirst = (lm < 0) ? lk : (lk < 0 ? lm : std::min(lm, lk));
          if (lfirst > 0) cost.s += 1;
          if (lm >= 0 && lk >= 0 && lk < lm) cost.l = 1;
          // R: blocks K and N
          long rk = pos(R, K), rn = pos(R, Nn);
          long rfirst = (rk < 0) ? rn : (rn < 0 ? rk : std::min(rk, rn));
          if (rfirst > 0) cost.s += 1;
          const int r = (rk >= 0 && rn >= 0 && rn < rk) ? 1 : 0;
          cost.lr = cost.l + r;
          cost.negf = -(int64_t)(M.size() + Nn.size() + K.size());
          if (!found || cost < best) {
            best = cost;
            found = true;
          }
        }
  }
  return best;
}

// -------------------------------------------------------- strength reduction + DP
namespace {

struct SubsetTerm {
  BPat pat;                 // after early summation, natural order
  std::string prod_idx, sum_idx;
  int64_t cost = -1;        // best total cost of building this subset's term
  int64_t mult = 0, sumc = 0;
  unsigned split = 0;       // left part of the best split (0 for leaves)
};

std::string indices_outside(const Expression& e, const Term& t, unsigned subset) {
  std::string keep = e.lhs_idx;
  for (size_t i = 0; i < t.factors.size(); ++i)
    if (!(subset >> i & 1u)) keep += t.factors[i].idx;
  return keep;
}

std::vector<std::string> permutations_of(std::string s) {
  std::sort(s.begin(), s.end());
  std::vector<std::string> out;
  do out.push_back(s);
  while (std::next_permutation(s.begin(), s.end()));
  return out;
}

}  // namespace

TermPlan plan_term(const Expression& e, int ti, const std::vector<TensorInfo>& tensors) {
  const Term& t = e.terms[ti];
  const int n = (int)t.factors.size();
  TermPlan tp;
  tp.scalar = t.scalar;
  tp.eq = eqspp(t, tensors);
  const unsigned full = (1u << n) - 1u;
  std::vector<SubsetTerm> st(full + 1);
  // leaves
  for (int i = 0; i < n; ++i) {
    SubsetTerm& s = st[1u << i];
    BPat p = tp.eq[i];
    s.prod_idx = p.idx;
    BPat q = sum_out(p, indices_outside(e, t, 1u << i));
    for (char c : p.idx)
      if (q.idx.find(c) == std::string::npos) s.sum_idx.push_back(c);
    s.sumc = p.nnz() - q.nnz();
    s.cost = s.sumc;
    s.pat = q;
  }
  // subsets in increasing size: minimise over splits that keep the lowest factor left
  for (unsigned S = 1; S <= full; ++S) {
    if ((S & (S - 1)) == 0) continue;
    const unsigned low = S & (~S + 1u);
    const unsigned rest = S ^ low;
    const std::string keep = indices_outside(e, t, S);
    for (unsigned sub = rest;; sub = (sub - 1) & rest) {
      const unsigned A = low | sub, Bm = S ^ A;
      if (Bm != 0 && st[A].cost >= 0 && st[Bm].cost >= 0 &&
          product_volume(st[A].pat, st[Bm].pat) <= kMaxPatternSize) {
        BPat prod = product(st[A].pat, st[Bm].pat);
        BPat red = sum_out(prod, keep);
        const int64_t mult = prod.nnz(), sumc = prod.nnz() - red.nnz();
        const int64_t total = st[A].cost + st[Bm].cost + mult + sumc;
        if (st[S].cost < 0 || total < st[S].cost) {
          st[S].cost = total;
          st[S].mult = mult;
          st[S].sumc = sumc;
          st[S].split = A;
          st[S].prod_idx = prod.idx;
          st[S].sum_idx.clear();
          for (char c : prod.idx)
            if (red.idx.find(c) == std::string::npos) st[S].sum_idx.push_back(c);
          st[S].pat = red;
        }
      }
      if (sub == 0) break;
    }
  }
  if (st[full].cost < 0) throw Error(YT_ERR_UNSUPPORTED, "every contraction order needs an intermediate above 2^24 entries");
  tp.nz_cost = st[full].cost;
  {
    // naive: one n-ary product over the whole index space, then one summation
    // (-1 when that space is above the planner's size limit)
    BPat all = tp.eq[0];
    bool small = true;
    for (int i = 1; i < n && small; ++i) {
      if (product_volume(all, tp.eq[i]) > kMaxPatternSize) small = false;
      else all = product(all, tp.eq[i]);
    }
    if (small) {
      BPat red = sum_out(all, e.lhs_idx);
      tp.naive_cost = (int64_t)(n - 1) * all.nnz() + (all.nnz() - red.nnz());
    } else {
      tp.naive_cost = -1;
    }
  }
  // tree in post-order
  std::function<int(unsigned)> emit = [&](unsigned S) -> int {
    Node nd;
    if ((S & (S - 1)) == 0) {
      int i = 0;
      while (!(S >> i & 1u)) ++i;
      nd.factor = i;
    } else {
      nd.left = emit(st[S].split);
      nd.right = emit(S ^ st[S].split);
    }
    nd.prod_idx = st[S].prod_idx;
    nd.sum_idx = st[S].sum_idx;
    nd.pat = st[S].pat;
    nd.mult_cost = st[S].mult;
    nd.sum_cost = st[S].sumc;
    tp.nodes.push_back(nd);
    return (int)tp.nodes.size() - 1;
  };
  emit(full);

  // permutation DP (post-order); permissible orders: all permutations of an internal
  // node's result (up to 7 indices), the fixed order of a leaf, the LHS order at the root
  const int root = (int)tp.nodes.size() - 1;
  std::vector<std::vector<std::string>> P(tp.nodes.size());
  std::vector<std::map<std::string, LogCost>> F(tp.nodes.size());
  std::vector<std::map<std::string, std::pair<std::string, std::string>>> arg(tp.nodes.size());
  for (int v = 0; v <= root; ++v) {
    Node& nd = tp.nodes[v];
    if (v == root) {
      P[v] = {e.lhs_idx};
    } else if (nd.left < 0) {
      P[v] = {nd.pat.idx};
    } else if (nd.pat.idx.size() <= 7) {
      P[v] = permutations_of(nd.pat.idx);
    } else {
      P[v] = {nd.pat.idx};
    }
    for (const std::string& xv : P[v]) {
      if (nd.left < 0) {
        F[v][xv] = LogCost{};
        continue;
      }
      bool have = false;
      LogCost best;
      std::pair<std::string, std::string> barg;
      for (const std::string& xl : P[nd.left])
        for (const std::string& xr : P[nd.right]) {
          const LogCost c = min_log(xv, xl, xr) + F[nd.left][xl] + F[nd.right][xr];
          if (!have || c < best) {
            best = c;
            barg = {xl, xr};
            have = true;
          }
        }
      F[v][xv] = best;
      arg[v][xv] = barg;
    }
  }
  tp.log_cost = F[root][e.lhs_idx];
  // assign the chosen orders top-down and describe the tree
  std::function<std::string(int, const std::string&)> assign = [&](int v, const std::string& x) -> std::string {
    Node& nd = tp.nodes[v];
    nd.pat = permute(nd.pat, x);
    std::string label;
    if (nd.left < 0) {
      label = tensors[t.factors[nd.factor].tensor].name + "[" + t.factors[nd.factor].idx + "]";
      if (!nd.sum_idx.empty()) label = "sum_" + nd.sum_idx + "(" + label + ")";
      return label;
    }
    const auto& a = arg[v].at(x);
    std::string l = assign(nd.left, a.first), r = assign(nd.right, a.second);
    label = "(" + l + "*" + r + ")";
    if (!nd.sum_idx.empty()) label = "sum_" + nd.sum_idx + label;
    return label + "[" + x + "]";
  };
  tp.order = assign(root, e.lhs_idx);
  return tp;
}

}  // namespace plan
}  // namespace yt
