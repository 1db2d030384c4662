// C ABI of the planner and the batched executor: yt_plan_create, yt_plan_stats_get,
// yt_plan_eqspp, yt_execute_batched, yt_plan_destroy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "common.h"
#include "executor.cuh"
#include "planner.h"

using namespace yt;
using namespace yt::plan;

struct yt_plan {
  std::vector<TensorInfo> tensors;
  Expression expr;
  std::vector<TermPlan> terms;
  yt_precision prec = YT_F64;
  std::vector<ExecOp> ops;
  std::vector<int> prog;
  std::vector<int> slot_of_tensor;     // per-element tensor index -> pointer slot
  int temp_entries = 1;
  bool element_per_warp = false;       // executor kernel, chosen at creation
  bool ew_global_temps = false;        // element per warp, temporaries in global scratch
  double nz_flops = 0, hw_flops = 0, naive_flops = 0;
  int64_t bytes_per_element = 0;
  int n_binary = 0;
  std::string order;
  // device copies
  ExecOp* d_ops = nullptr;            // device state below is created on first execution
  int* d_prog = nullptr;
  void* d_consts = nullptr;
  std::vector<int> const_offset;       // per tensor, offset into consts (globals)
  // host copy of the constants in the plan's precision (double or float values), built
  // at creation: the source of every upload, alive as long as the plan
  std::vector<unsigned char> consts_host;
  size_t n_consts = 0;
  // scratch for temporaries, grown on demand
  mutable std::mutex mu;
  mutable void* scratch = nullptr;
  mutable size_t scratch_bytes = 0;
  ~yt_plan() {
    if (d_ops) cudaFree(d_ops);
    if (d_prog) cudaFree(d_prog);
    if (d_consts) cudaFree(d_consts);
    if (scratch) cudaFree(scratch);
  }
};

namespace {

std::vector<size_t> strides(const std::vector<int>& dims) {
  std::vector<size_t> s(dims.size());
  size_t a = 1;
  for (size_t i = 0; i < dims.size(); ++i) { s[i] = a; a *= (size_t)dims[i]; }
  return s;
}

// Operand of an operation: where its values live and how its index string maps to
// offsets.
struct Operand {
  int kind = kOpNone, ref = 0, size = 0;
  std::string idx;             // storage order
  std::vector<int> dims;
  const BPat* pat = nullptr;   // non-zero pattern in storage order
};

// Appends one operation C = sum over `summed` of A * B (B may be absent) restricted to
// the non-zeros of the operands' patterns, grouped by output entry.
void emit_op(yt_plan* p, const Operand& C, const BPat& cpat, const Operand& A, const Operand* B,
             const std::string& summed, double scalar, bool accumulate, int kind) {
  // iteration space: output indices (C order) then summed indices
  std::string space = C.idx + summed;
  std::vector<int> dims = C.dims;
  std::map<char, int> size;
  for (size_t i = 0; i < A.idx.size(); ++i) size[A.idx[i]] = A.dims[i];
  if (B)
    for (size_t i = 0; i < B->idx.size(); ++i) size[B->idx[i]] = B->dims[i];
  for (char c : summed) dims.push_back(size.at(c));
  size_t vol = 1;
  for (int d : dims) vol *= (size_t)d;
  const auto sc = strides(C.dims), sa = strides(A.dims);
  std::vector<size_t> sb = B ? strides(B->dims) : std::vector<size_t>();
  std::vector<size_t> ma(space.size(), 0), mb(space.size(), 0), mc(space.size(), 0);
  for (size_t d = 0; d < space.size(); ++d) {
    auto pa = A.idx.find(space[d]);
    if (pa != std::string::npos) ma[d] = sa[pa];
    if (B) {
      auto pb = B->idx.find(space[d]);
      if (pb != std::string::npos) mb[d] = sb[pb];
    }
    if (d < C.idx.size()) mc[d] = sc[d];
  }
  std::map<int, std::vector<std::pair<int, int>>> rows;
  std::vector<int> i(dims.size(), 0);
  for (size_t lin = 0; lin < vol; ++lin) {
    size_t oa = 0, ob = 0, oc = 0;
    for (size_t d = 0; d < dims.size(); ++d) {
      oa += i[d] * ma[d];
      ob += i[d] * mb[d];
      oc += i[d] * mc[d];
    }
    if (cpat.bits[oc] && A.pat->bits[oa] && (!B || B->pat->bits[ob])) rows[(int)oc].push_back({(int)oa, (int)ob});
    for (size_t d = 0; d < dims.size(); ++d) {
      if (++i[d] < dims[d]) break;
      i[d] = 0;
    }
  }
  ExecOp op{};
  op.kind = kind;
  op.out_kind = C.kind; op.out_ref = C.ref; op.out_size = C.size;
  op.a_kind = A.kind; op.a_ref = A.ref; op.a_size = A.size;
  op.b_kind = B ? B->kind : kOpNone; op.b_ref = B ? B->ref : 0; op.b_size = B ? B->size : 0;
  op.scalar = scalar;
  op.accumulate = accumulate ? 1 : 0;
  op.nrows = (int)rows.size();
  op.rows_off = (int)p->prog.size();
  for (auto& kv : rows) p->prog.push_back(kv.first);
  op.rp_off = (int)p->prog.size();
  int cnt = 0;
  for (auto& kv : rows) { p->prog.push_back(cnt); cnt += (int)kv.second.size(); }
  p->prog.push_back(cnt);
  op.pairs_off = (int)p->prog.size();
  for (auto& kv : rows)
    for (auto& pr : kv.second) { p->prog.push_back(pr.first); p->prog.push_back(pr.second); }
  p->ops.push_back(op);
  p->hw_flops += 2.0 * cnt + (scalar != 1.0 ? op.nrows : 0) + (accumulate && C.kind == kOpTensor ? op.nrows : 0);
  if (kind == kOpProduct) p->n_binary += 1;
}

Operand tensor_operand(yt_plan* p, int tensor, const std::string& idx, const BPat* pat) {
  Operand o;
  const TensorInfo& t = p->tensors[tensor];
  o.idx = idx;
  o.dims = t.shape;
  o.size = 1;
  for (int d : t.shape) o.size *= d;
  o.pat = pat;
  if (t.global) { o.kind = kOpConst; o.ref = p->const_offset[tensor]; }
  else { o.kind = kOpTensor; o.ref = p->slot_of_tensor[tensor]; }
  return o;
}

void compile(yt_plan* p) {
  const Expression& e = p->expr;
  const int lhs = e.lhs;
  std::vector<uint8_t> dense_lhs_bits;
  BPat lhs_dense;
  lhs_dense.idx = e.lhs_idx;
  lhs_dense.dims = p->tensors[lhs].shape;
  size_t lhs_size = 1;
  for (int d : lhs_dense.dims) lhs_size *= (size_t)d;
  lhs_dense.bits.assign(lhs_size, 1);
  if (!e.accumulate) {
    ExecOp z{};
    z.kind = kOpZero;
    z.out_kind = kOpTensor;
    z.out_ref = p->slot_of_tensor[lhs];
    z.out_size = (int)lhs_size;
    z.scalar = 1.0;
    p->ops.push_back(z);
  }
  int max_temp = 1;
  for (size_t ti = 0; ti < p->terms.size(); ++ti) {
    TermPlan& tp = p->terms[ti];
    const Term& term = e.terms[ti];
    int temp_next = 0;
    std::vector<Operand> res(tp.nodes.size());
    const int root = (int)tp.nodes.size() - 1;
    for (int v = 0; v <= root; ++v) {
      Node& nd = tp.nodes[v];
      const bool is_root = v == root;
      Operand out;
      if (is_root) {
        out = tensor_operand(p, lhs, e.lhs_idx, &lhs_dense);
      } else {
        out.kind = kOpTemp;
        out.ref = temp_next;
        out.idx = nd.pat.idx;
        out.dims = nd.pat.dims;
        out.size = (int)nd.pat.size();
        out.pat = &nd.pat;
      }
      if (nd.left < 0) {
        const Factor& f = term.factors[nd.factor];
        Operand leaf = tensor_operand(p, f.tensor, f.idx, &tp.eq[nd.factor]);
        if (nd.sum_idx.empty() && !is_root) {
          res[v] = leaf;                         // used in place by its parent
          continue;
        }
        emit_op(p, out, nd.pat, leaf, nullptr, nd.sum_idx, is_root ? tp.scalar : 1.0, is_root, kOpUnary);
      } else {
        emit_op(p, out, nd.pat, res[nd.left], &res[nd.right], nd.sum_idx, is_root ? tp.scalar : 1.0,
                is_root, kOpProduct);
      }
      if (!is_root) {
        temp_next += out.size;
        res[v] = out;
      }
    }
    max_temp = std::max(max_temp, temp_next);
    p->nz_flops += (double)tp.nz_cost + (tp.scalar != 1.0 ? (double)tp.nodes[root].pat.nnz() : 0.0) +
                   (e.accumulate || ti > 0 ? (double)tp.nodes[root].pat.nnz() : 0.0);
    p->naive_flops = (tp.naive_cost < 0 || p->naive_flops < 0) ? -1.0 : p->naive_flops + (double)tp.naive_cost;
    if (!p->order.empty()) p->order += " + ";
    if (tp.scalar != 1.0) p->order += std::to_string(tp.scalar) + "*";
    p->order += tp.order;
  }
  p->temp_entries = max_temp;
  // kernel choice: one element per warp, the temporaries in shared memory when four
  // warps' temporaries fit in 96 KB (two blocks per SM at least), else in a global scratch
  // slice per warp (16 warps per SM; with one block per SM and shared-memory temporaries it
  // was slower than the lane-per-element kernel, with global ones 1.9x faster for the
  // order-6 fused-simulation chain).  Rows are reordered by decreasing number of products
  // (output entry order among equals), so that the lanes of a warp, which take
  // consecutive rows, run similar numbers of products.  The lane-per-element kernel (the
  // allocation-free entry point) reads the same rows in that order.
  const size_t word_bytes = p->prec == YT_F32 ? 4 : 8;
  p->element_per_warp = true;
  p->ew_global_temps = (size_t)kEwWarps * p->temp_entries * word_bytes > (size_t)kEwSmemCap;
  if (p->element_per_warp) {
    for (const ExecOp& op : p->ops) {
      if (op.kind == kOpZero || op.nrows == 0) continue;
      std::vector<int> idx(op.nrows);
      for (int r = 0; r < op.nrows; ++r) idx[r] = r;
      auto len = [&](int r) { return p->prog[op.rp_off + r + 1] - p->prog[op.rp_off + r]; };
      std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return len(a) > len(b); });
      std::vector<int> rows_new, rp_new(1, 0), pairs_new;
      for (int r : idx) {
        rows_new.push_back(p->prog[op.rows_off + r]);
        const int b = p->prog[op.rp_off + r], e = p->prog[op.rp_off + r + 1];
        for (int t = b; t < e; ++t) {
          pairs_new.push_back(p->prog[op.pairs_off + 2 * t]);
          pairs_new.push_back(p->prog[op.pairs_off + 2 * t + 1]);
        }
        rp_new.push_back((int)pairs_new.size() / 2);
      }
      std::copy(rows_new.begin(), rows_new.end(), p->prog.begin() + op.rows_off);
      std::copy(rp_new.begin(), rp_new.end(), p->prog.begin() + op.rp_off);
      std::copy(pairs_new.begin(), pairs_new.end(), p->prog.begin() + op.pairs_off);
    }
  }
  // bytes per element: per-element operands read once, result written (and read for +=)
  std::vector<bool> seen(p->tensors.size(), false);
  const size_t word = p->prec == YT_F32 ? 4 : 8;
  for (const Term& t : e.terms)
    for (const Factor& f : t.factors)
      if (!p->tensors[f.tensor].global && !seen[f.tensor]) {
        seen[f.tensor] = true;
        size_t s = 1;
        for (int d : p->tensors[f.tensor].shape) s *= (size_t)d;
        p->bytes_per_element += (int64_t)(s * word);
      }
  p->bytes_per_element += (int64_t)(lhs_size * word * (e.accumulate ? 2 : 1));
}

void assign_const_offsets(yt_plan* p) {
  p->const_offset.assign(p->tensors.size(), 0);
  int off = 0;
  for (size_t i = 0; i < p->tensors.size(); ++i)
    if (p->tensors[i].global) {
      p->const_offset[i] = off;
      off += (int)p->tensors[i].values.size();
    }
}

// The constants of all global tensors, in descriptor order, converted once to the plan's
// precision.
template <typename Real>
void pack_consts(yt_plan* p) {
  std::vector<Real> c;
  for (size_t i = 0; i < p->tensors.size(); ++i)
    if (p->tensors[i].global)
      for (double v : p->tensors[i].values) c.push_back((Real)v);
  p->n_consts = c.size();
  if (c.empty()) c.push_back(Real(0));
  p->consts_host.resize(c.size() * sizeof(Real));
  std::memcpy(p->consts_host.data(), c.data(), p->consts_host.size());
}

// Device copies of the constants and the operation list, made on first execution.
template <typename Real>
void ensure_device(yt_plan* p) {
  if (p->d_ops) return;
  cuda_check(cudaMalloc(&p->d_consts, p->consts_host.size()), "cudaMalloc consts");
  cuda_check(cudaMemcpy(p->d_consts, p->consts_host.data(), p->consts_host.size(), cudaMemcpyHostToDevice), "copy consts");
  cuda_check(cudaMalloc(&p->d_prog, std::max<size_t>(1, p->prog.size()) * sizeof(int)), "cudaMalloc prog");
  if (!p->prog.empty())
    cuda_check(cudaMemcpy(p->d_prog, p->prog.data(), p->prog.size() * sizeof(int), cudaMemcpyHostToDevice), "copy prog");
  ExecOp* d = nullptr;
  cuda_check(cudaMalloc(&d, std::max<size_t>(1, p->ops.size()) * sizeof(ExecOp)), "cudaMalloc ops");
  cuda_check(cudaMemcpy(d, p->ops.data(), p->ops.size() * sizeof(ExecOp), cudaMemcpyHostToDevice), "copy ops");
  p->d_ops = d;
}

template <typename Real>
void launch(yt_plan* p, void* const* ptrs, int64_t n, cudaStream_t st) {
  ExecPtrs<Real> T{};
  for (size_t i = 0; i < p->tensors.size(); ++i)
    if (!p->tensors[i].global) {
      YT_REQUIRE(ptrs[i] != nullptr, YT_ERR_INVALID, "null pointer for per-element tensor " + p->tensors[i].name);
      T.p[p->slot_of_tensor[i]] = static_cast<Real*>(ptrs[i]);
    }
  int dev = 0, sms = 0;
  cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
  // one element per warp with the temporaries in shared memory (kernel chosen at creation)
  const size_t ew_smem = (size_t)kEwWarps * p->temp_entries * sizeof(Real);
  if (p->element_per_warp && p->ew_global_temps) {
    // four blocks of four warps per SM, each warp's temporaries in its slice of the scratch
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n + kEwWarps - 1) / kEwWarps,
                                                                  (int64_t)sms * 4));
    const size_t need = (size_t)blocks * kEwWarps * p->temp_entries * sizeof(Real);
    std::lock_guard<std::mutex> lock(p->mu);
    ensure_device<Real>(p);
    if (p->scratch_bytes < need) {
      if (p->scratch) {
        cuda_check(cudaStreamSynchronize(st), "sync before scratch growth");
        cudaFree(p->scratch);
        p->scratch = nullptr;
        p->scratch_bytes = 0;
      }
      cuda_check(cudaMalloc(&p->scratch, need), "cudaMalloc scratch");
      p->scratch_bytes = need;
    }
    k_execute_ew<Real, true><<<(unsigned)blocks, kEwWarps * 32, 0, st>>>(
        p->d_ops, (int)p->ops.size(), p->d_prog, static_cast<const Real*>(p->d_consts), T,
        p->temp_entries, n, static_cast<Real*>(p->scratch));
    cuda_check(cudaGetLastError(), "k_execute_ew launch");
    return;
  }
  if (p->element_per_warp) {
    std::lock_guard<std::mutex> lock(p->mu);
    ensure_device<Real>(p);
    // the attribute belongs to the function, shared by all plans: always the cap, so that
    // plans launching from other threads never see a smaller value
    if (ew_smem > 48 * 1024)
      cuda_check(cudaFuncSetAttribute(k_execute_ew<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kEwSmemCap), "cudaFuncSetAttribute");
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n + kEwWarps - 1) / kEwWarps,
                                                                  (int64_t)sms * 16));
    k_execute_ew<Real><<<(unsigned)blocks, kEwWarps * 32, ew_smem, st>>>(
        p->d_ops, (int)p->ops.size(), p->d_prog, static_cast<const Real*>(p->d_consts), T,
        p->temp_entries, n);
    cuda_check(cudaGetLastError(), "k_execute_ew launch");
    return;
  }
  const int64_t tiles = (n + 31) / 32;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((tiles + 3) / 4, (int64_t)sms * 8));
  const size_t need = (size_t)blocks * 4 * p->temp_entries * 32 * sizeof(Real);
  std::lock_guard<std::mutex> lock(p->mu);
  ensure_device<Real>(p);
  if (p->scratch_bytes < need) {
    if (p->scratch) {
      cuda_check(cudaStreamSynchronize(st), "sync before scratch growth");
      cudaFree(p->scratch);
      p->scratch = nullptr;
      p->scratch_bytes = 0;
    }
    cuda_check(cudaMalloc(&p->scratch, need), "cudaMalloc scratch");
    p->scratch_bytes = need;
  }
  k_execute<Real><<<(unsigned)blocks, 128, 0, st>>>(p->d_ops, (int)p->ops.size(), p->d_prog,
                                                      static_cast<const Real*>(p->d_consts), T,
                                                      static_cast<Real*>(p->scratch), p->temp_entries, n);
  cuda_check(cudaGetLastError(), "k_execute launch");
}

}  // namespace

extern "C" yt_status yt_plan_create(const char* expr, const yt_tensor_desc* tensors,
                                    int32_t n_tensors, yt_precision precision, yt_plan** out) {
  return guarded([&] {
    YT_REQUIRE(out, YT_ERR_INVALID, "null out_plan");
    *out = nullptr;
    YT_REQUIRE(expr && tensors && n_tensors > 0, YT_ERR_INVALID, "null argument");
    YT_REQUIRE(precision == YT_F64 || precision == YT_F32, YT_ERR_UNSUPPORTED, "precision: YT_F64 or YT_F32");
    auto p = std::make_unique<yt_plan>();
    p->prec = precision;
    int slots = 0;
    for (int i = 0; i < n_tensors; ++i) {
      const yt_tensor_desc& d = tensors[i];
      YT_REQUIRE(d.name && d.ndim >= 0 && d.ndim <= 8, YT_ERR_INVALID, "tensor descriptor " + std::to_string(i));
      YT_REQUIRE(d.ndim == 0 || d.shape, YT_ERR_INVALID, "null shape");
      TensorInfo t;
      t.name = d.name;
      size_t sz = 1;
      for (int k = 0; k < d.ndim; ++k) {
        YT_REQUIRE(d.shape[k] > 0 && d.shape[k] <= 4096, YT_ERR_SHAPE, "dimension sizes must be 1..4096");
        t.shape.push_back(d.shape[k]);
        sz *= (size_t)d.shape[k];
      }
      YT_REQUIRE(sz <= (size_t(1) << 24), YT_ERR_UNSUPPORTED, "tensor too large");
      t.pattern.assign(sz, 1);
      if (d.pattern)
        for (size_t k = 0; k < sz; ++k) t.pattern[k] = d.pattern[k] ? 1 : 0;
      if (d.values) {
        t.global = true;
        t.values.assign(d.values, d.values + sz);
        for (size_t k = 0; k < sz; ++k)
          if (t.values[k] == 0.0) t.pattern[k] = 0;       // a known zero is a structural zero
      }
      for (const auto& o : p->tensors)
        YT_REQUIRE(o.name != t.name, YT_ERR_INVALID, "duplicate tensor name " + t.name);
      p->tensors.push_back(t);
      p->slot_of_tensor.push_back(t.global ? -1 : slots);
      if (!t.global) ++slots;
    }
    YT_REQUIRE(slots <= kMaxExecTensors, YT_ERR_UNSUPPORTED, "at most 16 per-element tensors");
    p->expr = parse(expr, p->tensors);
    for (size_t t = 0; t < p->expr.terms.size(); ++t) p->terms.push_back(plan_term(p->expr, (int)t, p->tensors));
    assign_const_offsets(p.get());
    if (precision == YT_F64) pack_consts<double>(p.get());
    else pack_consts<float>(p.get());
    compile(p.get());
    *out = p.release();
  });
}

extern "C" yt_status yt_plan_stats_get(const yt_plan* p, yt_plan_stats* s) {
  return guarded([&] {
    YT_REQUIRE(p && s, YT_ERR_INVALID, "null argument");
    std::memset(s, 0, sizeof(*s));
    s->nz_flops = p->nz_flops;
    s->hw_flops = p->hw_flops;
    s->naive_flops = p->naive_flops;
    s->bytes_per_element = p->bytes_per_element;
    s->n_ops = p->n_binary;
    s->n_terms = (int32_t)p->terms.size();
    LogCost lc;
    for (const auto& t : p->terms) lc = lc + t.log_cost;
    s->log_cost[0] = lc.s;
    s->log_cost[1] = lc.lr;
    s->log_cost[2] = lc.negf;
    s->log_cost[3] = lc.l;
    std::strncpy(s->order, p->order.c_str(), sizeof(s->order) - 1);
  });
}

extern "C" yt_status yt_plan_eqspp(const yt_plan* p, int32_t term, int32_t tensor_index, uint8_t* out) {
  return guarded([&] {
    YT_REQUIRE(p && out, YT_ERR_INVALID, "null argument");
    YT_REQUIRE(term >= 0 && term < (int)p->terms.size(), YT_ERR_INVALID, "term out of range");
    const Term& t = p->expr.terms[term];
    for (size_t f = 0; f < t.factors.size(); ++f)
      if (t.factors[f].tensor == tensor_index) {
        const BPat& b = p->terms[term].eq[f];
        std::memcpy(out, b.bits.data(), b.bits.size());
        return;
      }
    throw Error(YT_ERR_INVALID, "tensor does not occur in this term");
  });
}

extern "C" yt_status yt_execute_batched(const yt_plan* p, void* const* element_tensors,
                                        int64_t n_elements, yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(p && element_tensors, YT_ERR_INVALID, "null argument");
    YT_REQUIRE(n_elements >= 0, YT_ERR_INVALID, "negative element count");
    if (n_elements == 0) return;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    yt_plan* mp = const_cast<yt_plan*>(p);   // lazily created device state, under mp->mu
    if (p->prec == YT_F64) launch<double>(mp, element_tensors, n_elements, st);
    else launch<float>(mp, element_tensors, n_elements, st);
  });
}

extern "C" void yt_plan_destroy(yt_plan* p) { delete p; }

// ------------------------------------------------------ allocation-free execution
// yt_execute_batched_noalloc computes what yt_execute_batched computes, but every device
// buffer it needs lives in the fixed-size file-scope arrays below, so the call never
// allocates device memory.  It always runs the lane-per-element executor kernel
// (k_execute) with its temporaries in the fixed global scratch, also for the plans that
// yt_execute_batched runs on the element-per-warp kernel (k_execute_ew, temporaries in
// shared memory): that kernel needs a dynamic shared-memory size attribute set on the
// function beyond 48 KB, which this entry point leaves alone.  Results agree with
// yt_execute_batched up to the summation order; speed and the kernel named by a profiler
// can differ.  The arrays are reserved on every device that loads this library and stay
// reserved until the process exits.  All calls share them: each call first copies the
// plan's operation list, index lists and constants into them (from host copies owned by
// the plan), and the temporaries are written before they are read, so nothing has to
// start at zero.  Two calls whose work overlaps on the device (different streams, or
// devices sharing nothing but this process) race on these arrays.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // temporaries: 32 MiB
constexpr size_t kNoAllocProgInts = size_t(1) << 20;        // index lists: 4 MiB
constexpr size_t kNoAllocOps = 4096;                         // operations: 256 KiB
constexpr size_t kNoAllocConstDoubles = size_t(1) << 18;    // constants: 2 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static __device__ __align__(256) int g_noalloc_prog[kNoAllocProgInts];
static __device__ __align__(256) ExecOp g_noalloc_ops[kNoAllocOps];
static __device__ __align__(256) double g_noalloc_consts[kNoAllocConstDoubles];

// Device addresses of the arrays, looked up once per device with that device current.
struct NoAllocAddrs {
  bool ready = false;
  void* scratch = nullptr;
  void* prog = nullptr;
  void* ops = nullptr;
  void* consts = nullptr;
};
std::mutex g_noalloc_mu;
NoAllocAddrs g_noalloc_addrs[64];

NoAllocAddrs noalloc_addrs(int dev) {
  YT_REQUIRE(dev >= 0 && dev < 64, YT_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocAddrs& a = g_noalloc_addrs[dev];
  if (!a.ready) {
    cuda_check(cudaGetSymbolAddress(&a.scratch, g_noalloc_scratch), "cudaGetSymbolAddress(scratch)");
    cuda_check(cudaGetSymbolAddress(&a.prog, g_noalloc_prog), "cudaGetSymbolAddress(prog)");
    cuda_check(cudaGetSymbolAddress(&a.ops, g_noalloc_ops), "cudaGetSymbolAddress(ops)");
    cuda_check(cudaGetSymbolAddress(&a.consts, g_noalloc_consts), "cudaGetSymbolAddress(consts)");
    a.ready = true;
  }
  return a;
}

template <typename Real>
void launch_noalloc(const yt_plan* p, void* const* ptrs, int64_t n, cudaStream_t st) {
  // limits first: a request beyond the fixed arrays is an error, never a partial run
  const size_t per_warp = (size_t)p->temp_entries * 32 * sizeof(Real);
  const size_t slots = kNoAllocScratchBytes / per_warp;
  YT_REQUIRE(slots >= 4, YT_ERR_UNSUPPORTED,
             "plan temporaries need " + std::to_string(per_warp * 4) + " bytes per block; the "
             "allocation-free scratch holds " + std::to_string(kNoAllocScratchBytes));
  YT_REQUIRE(p->prog.size() <= kNoAllocProgInts, YT_ERR_UNSUPPORTED,
             "plan index lists exceed the allocation-free limit of 2^20 integers");
  YT_REQUIRE(p->ops.size() <= kNoAllocOps, YT_ERR_UNSUPPORTED,
             "plan has more than 4096 operations");
  YT_REQUIRE(p->n_consts * sizeof(Real) <= kNoAllocConstDoubles * sizeof(double), YT_ERR_UNSUPPORTED,
             "plan constants exceed the allocation-free limit of 2 MiB");
  ExecPtrs<Real> T{};
  for (size_t i = 0; i < p->tensors.size(); ++i)
    if (!p->tensors[i].global) {
      YT_REQUIRE(ptrs[i] != nullptr, YT_ERR_INVALID, "null pointer for per-element tensor " + p->tensors[i].name);
      T.p[p->slot_of_tensor[i]] = static_cast<Real*>(ptrs[i]);
    }
  int dev = 0, sms = 0;
  cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
  const NoAllocAddrs a = noalloc_addrs(dev);
  if (!p->prog.empty())
    cuda_check(cudaMemcpyAsync(a.prog, p->prog.data(), p->prog.size() * sizeof(int), cudaMemcpyHostToDevice, st), "copy prog");
  if (!p->ops.empty())
    cuda_check(cudaMemcpyAsync(a.ops, p->ops.data(), p->ops.size() * sizeof(ExecOp), cudaMemcpyHostToDevice, st), "copy ops");
  if (p->n_consts > 0)
    cuda_check(cudaMemcpyAsync(a.consts, p->consts_host.data(), p->n_consts * sizeof(Real), cudaMemcpyHostToDevice, st),
               "copy consts");
  const int64_t tiles = (n + 31) / 32;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>({(tiles + 3) / 4, (int64_t)sms * 8, (int64_t)(slots / 4)}));
  k_execute<Real><<<(unsigned)blocks, 128, 0, st>>>(static_cast<const ExecOp*>(a.ops), (int)p->ops.size(),
                                                      static_cast<const int*>(a.prog),
                                                      static_cast<const Real*>(a.consts), T,
                                                      static_cast<Real*>(a.scratch), p->temp_entries, n);
  cuda_check(cudaGetLastError(), "k_execute launch");
}

}  // namespace

extern "C" yt_status yt_execute_batched_noalloc(const yt_plan* p, void* const* element_tensors,
                                                int64_t n_elements, yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(p && element_tensors, YT_ERR_INVALID, "null argument");
    YT_REQUIRE(n_elements >= 0, YT_ERR_INVALID, "negative element count");
    if (n_elements == 0) return;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (p->prec == YT_F64) launch_noalloc<double>(p, element_tensors, n_elements, st);
    else launch_noalloc<float>(p, element_tensors, n_elements, st);
  });
}
