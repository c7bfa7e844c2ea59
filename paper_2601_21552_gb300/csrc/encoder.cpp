// encoder.cpp -- host bit-blaster: query IR (expression trees + constraints
// of Sec. V-A/V-B) -> equisatisfiable 3-CNF.
//
// The paper hands its integer constraints to a CP-SAT solver (Sec. V-B,
// step 10). Here each query is instead lowered to CNF so that the whole batch
// can be decided by the GPU DPLL. Every clause has at most three literals,
// which lets the device keep a clause inline in its occurrence entries.
//
// Gadgets (all Tseitin equivalences, constants folded, structurally hashed):
//   AND / XOR            3 / 4 clauses, one fresh variable
//   MAJ(a,b,c)           6 clauses (full-adder carry, comparator borrow)
//   full adder           sum = (a ^ b) ^ c, carry = MAJ(a, b, c)
//   a + b                ripple carry, exact width max(wa, wb) + 1
//   a * b (var x var)    AND partial products compressed column by column
//                        (full/half adders), exact width wa + wb
//   a * k (constant)     only the set bits of k contribute partial rows
//   a < b                borrow chain of a - b: b_{i+1} = MAJ(!a_i, b_i, b_i')
//   a == b (asserted)    two binary clauses per bit, no fresh variables
//   a / k, a % k         q, r fresh with a = k*q + r and r < k; shifts/masks
//                        when k is a power of two
//   a mod 2^k, ~a        C's unsigned k-bit wrap-around: the low k bits, and
//                        their negations; no clauses
// Input words get the lowest variable ids, most significant bit first, so a
// lowest-id tie break branches on inputs from the top bit down.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "scuba_internal.h"

namespace scuba {
namespace {

constexpr int64_t kMagic = 0x53435542LL;
constexpr int64_t kVersion = 1;
enum Op : int64_t {
  kFree = 1, kConst = 2, kAdd = 3, kMul = 4, kUlt = 5, kUle = 6, kEq = 7,
  kOr = 8, kAnd = 9, kNot = 10, kUdiv = 11, kUrem = 12,
  kTrunc = 13, kNotw = 14  // second field: a bit count in [1, 64]
};

// Literals are DIMACS ints; TRUE/FALSE constants are the two sentinels.
constexpr int kTrue = 0x40000000;
constexpr int kFalse = -0x40000000;
inline bool is_const(int l) { return l == kTrue || l == kFalse; }

struct Builder {
  int nvars = 0;
  std::vector<int64_t> cb{0};
  std::vector<int32_t> lits;

  int fresh() { return ++nvars; }
  void clause(std::initializer_list<int> ls) {
    for (int l : ls) lits.push_back(l);
    cb.push_back((int64_t)lits.size());
  }
  void empty_clause() { cb.push_back((int64_t)lits.size()); }

  static uint64_t key(int tag, int a, int b, int c = 0) {
    uint64_t h = (uint64_t)(uint32_t)tag * 0x9E3779B97F4A7C15ULL;
    h ^= (uint64_t)(uint32_t)a + 0x7F4A7C15ULL + (h << 6) + (h >> 2);
    h ^= (uint64_t)(uint32_t)b * 0xC2B2AE3D27D4EB4FULL + (h << 6) + (h >> 2);
    h ^= (uint64_t)(uint32_t)c * 0x165667B19E3779F9ULL + (h << 6) + (h >> 2);
    return h;
  }
  // memo keys may collide in principle; store the operands next to the result
  struct Entry { int tag, a, b, c, out; };
  std::unordered_map<uint64_t, std::vector<Entry>> table;
  int lookup(int tag, int a, int b, int c) {
    auto it = table.find(key(tag, a, b, c));
    if (it == table.end()) return 0;
    for (auto& e : it->second)
      if (e.tag == tag && e.a == a && e.b == b && e.c == c) return e.out;
    return 0;
  }
  void remember(int tag, int a, int b, int c, int out) {
    table[key(tag, a, b, c)].push_back({tag, a, b, c, out});
  }

  int AND(int a, int b) {
    if (a == kFalse || b == kFalse) return kFalse;
    if (a == kTrue) return b;
    if (b == kTrue) return a;
    if (a == b) return a;
    if (a == -b) return kFalse;
    if (a > b) std::swap(a, b);
    if (int z = lookup(1, a, b, 0)) return z;
    int z = fresh();
    clause({-z, a});
    clause({-z, b});
    clause({z, -a, -b});
    remember(1, a, b, 0, z);
    return z;
  }
  int OR(int a, int b) { return -AND(-a, -b); }
  int XOR(int a, int b) {
    if (is_const(a)) std::swap(a, b);
    if (b == kFalse) return a;
    if (b == kTrue) return -a;
    if (a == b) return kFalse;
    if (a == -b) return kTrue;
    // normalise polarity: xor(-a, b) = -xor(a, b)
    bool flip = false;
    if (a < 0) { a = -a; flip = !flip; }
    if (b < 0) { b = -b; flip = !flip; }
    if (a > b) std::swap(a, b);
    int z = lookup(2, a, b, 0);
    if (!z) {
      z = fresh();
      clause({-z, a, b});
      clause({-z, -a, -b});
      clause({z, -a, b});
      clause({z, a, -b});
      remember(2, a, b, 0, z);
    }
    return flip ? -z : z;
  }
  int MAJ(int a, int b, int c) {
    // constant inputs reduce to AND / OR
    if (is_const(a)) std::swap(a, c);
    if (is_const(b)) std::swap(b, c);
    if (c == kFalse) return AND(a, b);
    if (c == kTrue) return OR(a, b);
    if (a == b) return a;
    if (a == c) return a;
    if (b == c) return b;
    if (a == -b) return c;
    if (a == -c) return b;
    if (b == -c) return a;
    int s[3] = {a, b, c};
    std::sort(s, s + 3);
    if (int z = lookup(3, s[0], s[1], s[2])) return z;
    int z = fresh();
    clause({-a, -b, z});
    clause({-a, -c, z});
    clause({-b, -c, z});
    clause({a, b, -z});
    clause({a, c, -z});
    clause({b, c, -z});
    remember(3, s[0], s[1], s[2], z);
    return z;
  }
  void assert_lit(int l) {
    if (l == kTrue) return;
    if (l == kFalse) { empty_clause(); return; }
    clause({l});
  }
};

using Word = std::vector<int>;  // LSB first

int bit(const Word& w, size_t i) { return i < w.size() ? w[i] : kFalse; }

Word add(Builder& B, const Word& a, const Word& b) {
  size_t W = std::max(a.size(), b.size()) + 1;
  Word s(W, kFalse);
  int carry = kFalse;
  for (size_t i = 0; i < W; i++) {
    int x = bit(a, i), y = bit(b, i);
    s[i] = B.XOR(B.XOR(x, y), carry);
    carry = B.MAJ(x, y, carry);
  }
  return s;
}

// Exact product by column compression of the partial products.
Word mul(Builder& B, const Word& a, const Word& b) {
  size_t W = a.size() + b.size();
  std::vector<std::vector<int>> col(W + 1);
  for (size_t i = 0; i < a.size(); i++)
    for (size_t j = 0; j < b.size(); j++) {
      int p = B.AND(a[i], b[j]);
      if (p != kFalse) col[i + j].push_back(p);
    }
  Word out(W, kFalse);
  for (size_t c = 0; c < W; c++) {
    auto& v = col[c];
    size_t head = 0;
    while (v.size() - head > 1) {
      if (v.size() - head >= 3) {
        int x = v[head], y = v[head + 1], z = v[head + 2];
        head += 3;
        int s = B.XOR(B.XOR(x, y), z);
        int cy = B.MAJ(x, y, z);
        if (s != kFalse) v.push_back(s);
        if (cy != kFalse) col[c + 1].push_back(cy);
      } else {
        int x = v[head], y = v[head + 1];
        head += 2;
        int s = B.XOR(x, y);
        int cy = B.AND(x, y);
        if (s != kFalse) v.push_back(s);
        if (cy != kFalse) col[c + 1].push_back(cy);
      }
    }
    out[c] = (v.size() - head == 1) ? v[head] : kFalse;
  }
  return out;  // the product fits in W bits, so col[W] only holds FALSE carries
}

// a < b: borrow out of a - b over the common width
int ult(Builder& B, const Word& a, const Word& b) {
  size_t W = std::max(a.size(), b.size());
  int borrow = kFalse;
  for (size_t i = 0; i < W; i++) borrow = B.MAJ(-bit(a, i), bit(b, i), borrow);
  return borrow;
}

int eq(Builder& B, const Word& a, const Word& b) {
  size_t W = std::max(a.size(), b.size());
  int all = kTrue;
  for (size_t i = 0; i < W; i++) all = B.AND(all, -B.XOR(bit(a, i), bit(b, i)));
  return all;
}

Word constant(uint64_t v) {
  Word w;
  do {
    w.push_back((v & 1) ? kTrue : kFalse);
    v >>= 1;
  } while (v);
  return w;
}

struct Encoder {
  const int64_t* node;
  int64_t n;
  Builder B;
  std::vector<Word> word;
  std::vector<int> boolean;
  std::vector<int> bool_ready;
  // q, r of each (operand, divisor) pair, shared between UDIV and UREM
  std::unordered_map<uint64_t, std::pair<Word, Word>> divs;

  void assert_word_eq(const Word& a, const Word& b) {
    size_t W = std::max(a.size(), b.size());
    for (size_t i = 0; i < W; i++) {
      int x = bit(a, i), y = bit(b, i);
      if (is_const(x) && is_const(y)) {
        if (x != y) B.empty_clause();
      } else if (is_const(x)) {
        B.assert_lit(x == kTrue ? y : -y);
      } else if (is_const(y)) {
        B.assert_lit(y == kTrue ? x : -x);
      } else if (x != y) {
        B.clause({-x, y});
        B.clause({x, -y});
      }
    }
  }

  std::pair<Word, Word>& divide(int64_t x, uint64_t k) {
    uint64_t key = (uint64_t)x * 0x100000001ULL ^ k;
    auto it = divs.find(key);
    if (it != divs.end()) return it->second;
    const Word& a = word[x];
    Word q, r;
    if ((k & (k - 1)) == 0) {  // power of two: shift and mask
      int s = 0;
      while ((1ULL << s) < k) s++;
      for (size_t i = s; i < a.size(); i++) q.push_back(a[i]);
      if (q.empty()) q.push_back(kFalse);
      for (int i = 0; i < s; i++) r.push_back(bit(a, i));
      if (r.empty()) r.push_back(kFalse);
    } else {
      q.resize(a.size());
      for (auto& b : q) b = B.fresh();
      int wr = 0;
      while ((1ULL << wr) < k) wr++;
      r.resize(wr);
      for (auto& b : r) b = B.fresh();
      Word kq = mul(B, constant(k), q);
      Word sum = add(B, kq, r);
      assert_word_eq(sum, a);
      B.assert_lit(ult(B, r, constant(k)));
    }
    return divs[key] = {q, r};
  }

  int run(const int64_t* roots, int64_t r, std::vector<int32_t>& in_map,
          std::vector<int32_t>& widths) {
    word.assign(n, Word());
    boolean.assign(n, 0);
    // input words first, MSB with the lowest id
    for (int64_t i = 0; i < n; i++) {
      if (node[4 * i] != kFree) continue;
      int w = (int)node[4 * i + 1];
      int base = B.nvars;
      B.nvars += w;
      Word v(w);
      for (int k = 0; k < w; k++) v[k] = base + (w - k);
      word[i] = v;
      widths.push_back(w);
      for (int k = 0; k < w; k++) in_map.push_back(v[k]);
    }
    // asserted conjunctions are split and positive equalities are emitted
    // as bitwise equivalences; every other asserted node becomes a unit clause
    // on the output of its circuit
    std::vector<std::pair<int64_t, bool>> todo;
    for (int64_t k = 0; k < r; k++) todo.push_back({roots[k], true});
    std::vector<std::pair<int64_t, bool>> asserted;
    while (!todo.empty()) {
      auto [id, pol] = todo.back();
      todo.pop_back();
      int64_t op = node[4 * id];
      if (op == kNot) { todo.push_back({node[4 * id + 1], !pol}); continue; }
      if ((op == kAnd && pol) || (op == kOr && !pol)) {
        todo.push_back({node[4 * id + 1], pol});
        todo.push_back({node[4 * id + 2], pol});
        continue;
      }
      asserted.push_back({id, pol});
    }
    for (int64_t i = 0; i < n; i++) build(i);
    for (auto [id, pol] : asserted) {
      if (node[4 * id] == kEq && pol) {
        assert_word_eq(word[node[4 * id + 1]], word[node[4 * id + 2]]);
      } else {
        int b = boolean[id];
        B.assert_lit(pol ? b : -b);
      }
    }
    return 0;
  }

  void build(int64_t i) {
    int64_t op = node[4 * i], x = node[4 * i + 1], y = node[4 * i + 2];
    switch (op) {
      case kFree: break;
      case kConst: word[i] = constant((uint64_t)x); break;
      case kAdd: word[i] = add(B, word[x], word[y]); break;
      case kMul: word[i] = mul(B, word[x], word[y]); break;
      case kUdiv: word[i] = divide(x, (uint64_t)node[4 * y + 1]).first; break;
      case kUrem: word[i] = divide(x, (uint64_t)node[4 * y + 1]).second; break;
      case kTrunc:
        word[i].assign(word[x].begin(), word[x].begin() + std::min<size_t>(word[x].size(), y));
        if (word[i].empty()) word[i].push_back(kFalse);
        break;
      case kNotw:
        word[i].resize((size_t)y);
        for (int64_t k = 0; k < y; k++) word[i][k] = -bit(word[x], (size_t)k);
        break;
      case kUlt: boolean[i] = ult(B, word[x], word[y]); break;
      case kUle: boolean[i] = -ult(B, word[y], word[x]); break;
      case kEq: boolean[i] = eq(B, word[x], word[y]); break;
      case kOr: boolean[i] = B.OR(boolean[x], boolean[y]); break;
      case kAnd: boolean[i] = B.AND(boolean[x], boolean[y]); break;
      case kNot: boolean[i] = -boolean[x]; break;
    }
  }
};

// build() constructs every node's circuit, including equality circuits of EQ
// nodes that are only asserted positively (a few dead, definitional gates).

int validate(const int64_t* a, int64_t len) {
  if (!a || len < 4 || a[0] != kMagic || a[1] != kVersion) return -1;
  int64_t n = a[2], r = a[3];
  if (n < 0 || r < 0 || len != 4 + 4 * n + r) return -1;
  const int64_t* node = a + 4;
  for (int64_t i = 0; i < n; i++) {
    int64_t op = node[4 * i], x = node[4 * i + 1], y = node[4 * i + 2];
    bool word_op = op == kAdd || op == kMul || op == kUlt || op == kUle || op == kEq ||
                   op == kUdiv || op == kUrem;
    auto is_word = [&](int64_t j) {
      int64_t o = node[4 * j];
      return o == kFree || o == kConst || o == kAdd || o == kMul || o == kUdiv || o == kUrem ||
             o == kTrunc || o == kNotw;
    };
    if (op == kFree) {
      if (x < 1 || x > 64) return -1;
    } else if (op == kConst) {
      if (x < 0) return -1;
    } else if (op == kTrunc || op == kNotw) {
      if (x < 0 || x >= i || !is_word(x) || y < 1 || y > 64) return -1;
    } else if (op >= kAdd && op <= kUrem) {
      if (x < 0 || x >= i) return -1;
      if (op != kNot && (y < 0 || y >= i)) return -1;
      if (word_op) {
        if (!is_word(x) || !is_word(y)) return -1;
      } else {
        if (is_word(x) || (op != kNot && is_word(y))) return -1;
      }
      if ((op == kUdiv || op == kUrem) && (node[4 * y] != kConst || node[4 * y + 1] < 1))
        return -1;
    } else {
      return -1;
    }
  }
  for (int64_t k = 0; k < r; k++) {
    int64_t id = a[4 + 4 * n + k];
    if (id < 0 || id >= n) return -1;
    int64_t o = node[4 * id];
    if (o == kFree || o == kConst || o == kAdd || o == kMul || o == kUdiv || o == kUrem ||
        o == kTrunc || o == kNotw)
      return -1;
  }
  return 0;
}

}  // namespace

int encode_query(const int64_t* ir, int64_t len, HostCnf* out) {
  if (validate(ir, len)) return -1;
  Encoder E;
  E.node = ir + 4;
  E.n = ir[2];
  out->in_map.clear();
  out->widths.clear();
  E.run(ir + 4 + 4 * E.n, ir[3], out->in_map, out->widths);
  out->nvars = E.B.nvars;
  out->clause_begin = std::move(E.B.cb);
  out->lits = std::move(E.B.lits);
  return 0;
}

}  // namespace scuba
