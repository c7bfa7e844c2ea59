// verify.cpp -- host re-verification of SAT models against the original
// integer constraints (Sec. V-B: an OOB is reported when every constraint
// holds for some input; the decoded input words are that input).
//
// Values are exact unsigned integers of any width (base-2^32 limbs), so the
// check does not depend on the CNF encoding at all.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "scuba_internal.h"

namespace scuba {
namespace {

using Big = std::vector<uint32_t>;  // little-endian limbs, no trailing zeros

void trim(Big& a) {
  while (!a.empty() && a.back() == 0) a.pop_back();
}

Big from_u64(uint64_t v) {
  Big r;
  while (v) {
    r.push_back((uint32_t)v);
    v >>= 32;
  }
  return r;
}

int cmp(const Big& a, const Big& b) {
  if (a.size() != b.size()) return a.size() < b.size() ? -1 : 1;
  for (size_t i = a.size(); i-- > 0;)
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  return 0;
}

Big add(const Big& a, const Big& b) {
  Big r(std::max(a.size(), b.size()) + 1, 0);
  uint64_t carry = 0;
  for (size_t i = 0; i < r.size(); i++) {
    uint64_t s = carry;
    if (i < a.size()) s += a[i];
    if (i < b.size()) s += b[i];
    r[i] = (uint32_t)s;
    carry = s >> 32;
  }
  trim(r);
  return r;
}

Big mul(const Big& a, const Big& b) {
  if (a.empty() || b.empty()) return {};
  std::vector<uint64_t> acc(a.size() + b.size() + 1, 0);
  for (size_t i = 0; i < a.size(); i++) {
    uint64_t carry = 0;
    for (size_t j = 0; j < b.size(); j++) {
      uint64_t cur = acc[i + j] + (uint64_t)a[i] * b[j] + carry;
      acc[i + j] = cur & 0xffffffffULL;
      carry = cur >> 32;
    }
    size_t k = i + b.size();
    while (carry) {
      uint64_t cur = acc[k] + carry;
      acc[k] = cur & 0xffffffffULL;
      carry = cur >> 32;
      k++;
    }
  }
  Big r(acc.size());
  for (size_t i = 0; i < acc.size(); i++) r[i] = (uint32_t)acc[i];
  trim(r);
  return r;
}

// a / k and a % k for a constant 1 <= k < 2^62 by bitwise long division (the
// partial remainder stays below 2k < 2^63 and is kept in 128 bits anyway)
void divmod(const Big& a, uint64_t k, Big& q, Big& r) {
  size_t nbits = a.size() * 32;
  q.assign(a.size(), 0);
  unsigned __int128 rem = 0;
  for (size_t i = nbits; i-- > 0;) {
    rem = (rem << 1) | ((a[i / 32] >> (i % 32)) & 1u);
    if (rem >= k) {
      rem -= k;
      q[i / 32] |= 1u << (i % 32);
    }
  }
  trim(q);
  r = from_u64((uint64_t)rem);
}

// a mod 2^k (k <= 64): the low k bits
Big low_bits(const Big& a, int64_t k) {
  Big r(a.begin(), a.begin() + std::min<size_t>(a.size(), (size_t)(k + 31) / 32));
  if (k % 32 && r.size() == (size_t)(k + 31) / 32) r.back() &= (1u << (k % 32)) - 1;
  trim(r);
  return r;
}

}  // namespace

int verify_words(const int64_t* ir, int64_t len, const uint64_t* words, int64_t nwords) {
  if (!ir || len < 4 || ir[0] != 0x53435542LL || ir[1] != 1) return -1;
  int64_t n = ir[2], r = ir[3];
  if (n < 0 || r < 0 || len != 4 + 4 * n + r) return -1;
  const int64_t* node = ir + 4;
  std::vector<Big> w(n);
  std::vector<char> b(n, 0);
  int64_t fi = 0;
  for (int64_t i = 0; i < n; i++) {
    int64_t op = node[4 * i], x = node[4 * i + 1], y = node[4 * i + 2];
    bool imm = op == 13 || op == 14;  // TRUNC / NOTW: y is a bit count
    if (op != 1 && op != 2 && (x < 0 || x >= i || (op != 10 && !imm && (y < 0 || y >= i))))
      return -1;
    if (imm && (y < 1 || y > 64)) return -1;
    switch (op) {
      case 1: {  // FREE
        if (fi >= nwords || x < 1 || x > 64) return -1;
        uint64_t v = words[fi++];
        if (x < 64 && (v >> x)) return -1;
        w[i] = from_u64(v);
        break;
      }
      case 2: w[i] = from_u64((uint64_t)x); break;
      case 3: w[i] = add(w[x], w[y]); break;
      case 4: w[i] = mul(w[x], w[y]); break;
      case 11:
      case 12: {
        if (node[4 * y] != 2 || node[4 * y + 1] < 1) return -1;
        Big q, rem;
        divmod(w[x], (uint64_t)node[4 * y + 1], q, rem);
        w[i] = op == 11 ? q : rem;
        break;
      }
      case 13: w[i] = low_bits(w[x], y); break;
      case 14: {  // (2^y - 1) - (x mod 2^y), y <= 64
        uint64_t m = y == 64 ? ~0ULL : (1ULL << y) - 1;
        Big t = low_bits(w[x], y);
        uint64_t v = t.empty() ? 0 : t[0];
        if (t.size() > 1) v |= (uint64_t)t[1] << 32;
        w[i] = from_u64(m - v);
        break;
      }
      case 5: b[i] = cmp(w[x], w[y]) < 0; break;
      case 6: b[i] = cmp(w[x], w[y]) <= 0; break;
      case 7: b[i] = cmp(w[x], w[y]) == 0; break;
      case 8: b[i] = b[x] || b[y]; break;
      case 9: b[i] = b[x] && b[y]; break;
      case 10: b[i] = !b[x]; break;
      default: return -1;
    }
  }
  for (int64_t k = 0; k < r; k++) {
    int64_t id = ir[4 + 4 * n + k];
    if (id < 0 || id >= n) return -1;
    if (!b[id]) return 0;
  }
  return 1;
}

}  // namespace scuba
