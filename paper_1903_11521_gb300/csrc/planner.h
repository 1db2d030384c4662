// Planner of Einstein-notation tensor operations (Sec. 4 of the paper), host side.
#pragma once
#include <array>
#include <cstdint>
#include <string>
#include <vector>

namespace yt {
namespace plan {

// Boolean sparsity pattern over an ordered index string, column-major (first index
// fastest).
struct BPat {
  std::string idx;
  std::vector<int> dims;
  std::vector<uint8_t> bits;
  size_t size() const { return bits.size(); }
  int64_t nnz() const;
};

BPat product(const BPat& a, const BPat& b);                 // indices: a.idx then b's new ones
BPat sum_out(const BPat& v, const std::string& keep);       // OR over indices not in keep
BPat permute(const BPat& v, const std::string& order);      // reorder (same index set)

struct TensorInfo {
  std::string name;
  std::vector<int> shape;
  std::vector<uint8_t> pattern;     // column-major, prod(shape)
  bool global = false;              // constant values owned by the plan
  std::vector<double> values;       // global only
};

struct Factor {
  int tensor;        // index into tensors
  std::string idx;   // one letter per dimension
};

struct Term {
  double scalar = 1.0;
  std::vector<Factor> factors;
};

struct Expression {
  int lhs = -1;
  std::string lhs_idx;
  bool accumulate = false;
  std::vector<Term> terms;
};

// Parses "Q[kp] += 2.0 * A[kl] * B[lp] + C[kp]" against named tensors.  Throws
// yt::Error(YT_ERR_PARSE / YT_ERR_SHAPE / YT_ERR_INVALID).
Expression parse(const std::string& text, const std::vector<TensorInfo>& tensors);

// Equivalent sparsity patterns (Eq. compeqspp) of every factor of a term, in the
// factor's own index order.
std::vector<BPat> eqspp(const Term& term, const std::vector<TensorInfo>& tensors);

// LoG cost (s, l + r, -f, l) of Sec. 4.5.2, compared lexicographically.
struct LogCost {
  int64_t s = 0, lr = 0, negf = 0, l = 0;
  LogCost operator+(const LogCost& o) const { return {s + o.s, lr + o.lr, negf + o.negf, l + o.l}; }
  bool operator<(const LogCost& o) const {
    if (s != o.s) return s < o.s;
    if (lr != o.lr) return lr < o.lr;
    if (negf != o.negf) return negf < o.negf;
    return l < o.l;
  }
  bool operator==(const LogCost& o) const { return s == o.s && lr == o.lr && negf == o.negf && l == o.l; }
};

// Minimum LoG cost of C[c] = sum A[a] B[b] over all Loop-over-GEMM mappings (fused index
// groups M, N, K taken as runs of consecutive indices, both operand roles).
LogCost min_log(const std::string& c, const std::string& a, const std::string& b);

// Node of a strength-reduced binary tree.
struct Node {
  int left = -1, right = -1;    // children (internal node) or -1
  int factor = -1;              // leaf: factor index in the term
  std::string prod_idx;         // indices of the product before summation (internal)
  std::string sum_idx;          // indices summed at this node
  BPat pat;                     // result pattern (index order = chosen permutation)
  int64_t mult_cost = 0, sum_cost = 0;
};

struct TermPlan {
  double scalar = 1.0;
  std::vector<Node> nodes;      // post-order; last node is the root
  std::vector<BPat> eq;         // EQSPP per factor
  int64_t nz_cost = 0;          // strength-reduced sparse cost (Sec. 4.3)
  int64_t naive_cost = 0;
  LogCost log_cost;             // DP optimum over the temporaries' index orders
  std::string order;            // human-readable tree with chosen index orders
};

// Strength reduction (exhaustive over subsets) followed by the permutation DP
// (Eqs. permopt, permcost, subproblem).  The root's order is the LHS order.
TermPlan plan_term(const Expression& e, int term, const std::vector<TensorInfo>& tensors);

}  // namespace plan
}  // namespace yt
