// host_api.cpp -- host half of the C ABI: batch encoding on a thread pool,
// CSR packing, input maps, model re-verification and error reporting.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/scuba.h"
#include "scuba_internal.h"

namespace scuba {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

}  // namespace scuba

struct scuba_encoded {
  std::vector<scuba::HostCnf> cnf;
  bool released = false;  // clause storage freed; sizes/inputs/verify still work
  int64_t clauses = 0, lits = 0;
};

namespace {

int hw_threads(int32_t want) {
  int n = (int)std::thread::hardware_concurrency();
  if (n < 1) n = 1;
  if (want > 0) n = std::min<int>(want, 1024);
  return n;
}

template <class F>
void parallel_for(int n, int nthreads, F f) {
  std::atomic<int> next{0};
  auto body = [&]() {
    for (;;) {
      int i = next.fetch_add(1);
      if (i >= n) break;
      f(i);
    }
  };
  int t = std::max(1, std::min(nthreads, n));
  std::vector<std::thread> pool;
  for (int k = 1; k < t; k++) pool.emplace_back(body);
  body();
  for (auto& th : pool) th.join();
}

}  // namespace

extern "C" {

const char* scuba_last_error(void) { return scuba::g_err.c_str(); }

int scuba_version(void) { return 2; }

int scuba_encode_batch(int32_t n, const int64_t* irs, const int64_t* ir_offsets,
                       int32_t nthreads, scuba_encoded** out) {
  if (n < 0 || !out || (n > 0 && (!irs || !ir_offsets))) {
    scuba::set_error("scuba_encode_batch: bad arguments");
    return SCUBA_ERR_ARG;
  }
  scuba::NvtxRange range("scuba encode");
  scuba_encoded* enc = nullptr;
  try {
    enc = new scuba_encoded;
    enc->cnf.resize(n);
  } catch (...) {
    delete enc;
    scuba::set_error("scuba_encode_batch: out of host memory");
    return SCUBA_ERR_NOMEM;
  }
  // no exception may leave a pool thread (it would terminate the process):
  // a query whose circuit does not fit in host memory is reported instead
  std::atomic<int> bad{-1}, oom{-1};
  parallel_for(n, hw_threads(nthreads), [&](int i) {
    int64_t b = ir_offsets[i], e = ir_offsets[i + 1];
    int r;
    try {
      r = e < b ? -1 : scuba::encode_query(irs + b, e - b, &enc->cnf[i]);
    } catch (...) {  // the batch is discarded below
      int expect = -1;
      oom.compare_exchange_strong(expect, i);
      return;
    }
    if (r != 0) {
      int expect = -1;
      bad.compare_exchange_strong(expect, i);
    }
  });
  if (oom.load() >= 0) {
    scuba::set_error("scuba_encode_batch: out of host memory encoding query " +
                     std::to_string(oom.load()));
    delete enc;
    return SCUBA_ERR_NOMEM;
  }
  if (bad.load() >= 0) {
    scuba::set_error("scuba_encode_batch: malformed IR at query " + std::to_string(bad.load()));
    delete enc;
    return SCUBA_ERR_MALFORMED;
  }
  for (auto& c : enc->cnf) {
    enc->clauses += (int64_t)c.clause_begin.size() - 1;
    enc->lits += (int64_t)c.lits.size();
  }
  *out = enc;
  return SCUBA_OK;
}

int scuba_encoded_sizes(const scuba_encoded* enc, int64_t* s) {
  if (!enc || !s) return SCUBA_ERR_ARG;
  int64_t C = enc->clauses, L = enc->lits, V = 0, mx = 0, bits = 0;
  for (auto& c : enc->cnf) {
    V += c.nvars;
    mx = std::max<int64_t>(mx, c.nvars);
    bits += (int64_t)c.in_map.size();
  }
  s[0] = (int64_t)enc->cnf.size();
  s[1] = C;
  s[2] = L;
  s[3] = V;
  s[4] = mx;
  s[5] = bits;
  return SCUBA_OK;
}

int scuba_encoded_copy(const scuba_encoded* enc, int64_t* icb, int64_t* cb, int32_t* lits,
                       int32_t* nv, int64_t* vb) {
  if (!enc || !icb || !cb || !lits || !nv || !vb) return SCUBA_ERR_ARG;
  if (enc->released) {
    scuba::set_error("scuba_encoded_copy: clause storage was released");
    return SCUBA_ERR_ARG;
  }
  const int n = (int)enc->cnf.size();
  // offsets first (sequential prefix sums), then the bulk copy in parallel
  std::vector<int64_t> lit_base(n + 1, 0);
  icb[0] = 0;
  vb[0] = 0;
  for (int i = 0; i < n; i++) {
    const auto& c = enc->cnf[i];
    icb[i + 1] = icb[i] + (int64_t)c.clause_begin.size() - 1;
    lit_base[i + 1] = lit_base[i] + (int64_t)c.lits.size();
    nv[i] = c.nvars;
    vb[i + 1] = vb[i] + c.nvars;
  }
  cb[icb[n]] = lit_base[n];
  parallel_for(n, hw_threads(0), [&](int i) {
    const auto& c = enc->cnf[i];
    int64_t nc = (int64_t)c.clause_begin.size() - 1;
    for (int64_t k = 0; k < nc; k++) cb[icb[i] + k] = lit_base[i] + c.clause_begin[k];
    if (!c.lits.empty()) std::memcpy(lits + lit_base[i], c.lits.data(), c.lits.size() * 4);
  });
  return SCUBA_OK;
}

int scuba_encoded_inputs(const scuba_encoded* enc, int64_t* iib, int32_t* width, int32_t* var) {
  if (!enc || !iib || !width || !var) return SCUBA_ERR_ARG;
  int64_t words = 0, bits = 0;
  iib[0] = 0;
  for (size_t i = 0; i < enc->cnf.size(); i++) {
    const auto& c = enc->cnf[i];
    for (int32_t w : c.widths) width[words++] = w;
    for (int32_t v : c.in_map) var[bits++] = v;
    iib[i + 1] = words;
  }
  return SCUBA_OK;
}

void scuba_encoded_free(scuba_encoded* enc) { delete enc; }

int scuba_encoded_release_clauses(scuba_encoded* enc) {
  if (!enc) return SCUBA_ERR_ARG;
  for (auto& c : enc->cnf) {
    std::vector<int64_t>().swap(c.clause_begin);
    std::vector<int32_t>().swap(c.lits);
  }
  enc->released = true;
  return SCUBA_OK;
}

int scuba_verify_batch(const scuba_encoded* enc, const int64_t* irs, const int64_t* ir_offsets,
                       const uint8_t* verdict, const uint8_t* model, int32_t nthreads,
                       uint8_t* ok) {
  if (!enc || !irs || !ir_offsets || !verdict || !model || !ok) return SCUBA_ERR_ARG;
  scuba::NvtxRange range("scuba verify");
  const int n = (int)enc->cnf.size();
  std::vector<int64_t> vb(n + 1, 0);
  for (int i = 0; i < n; i++) vb[i + 1] = vb[i] + enc->cnf[i].nvars;
  std::atomic<int> fails{0};
  std::atomic<bool> oom{false};
  auto check = [&](int i) {
    if (verdict[i] != SCUBA_SAT) {
      ok[i] = 2;
      return;
    }
    const auto& c = enc->cnf[i];
    std::vector<uint64_t> words(c.widths.size(), 0);
    size_t off = 0;
    for (size_t w = 0; w < c.widths.size(); w++) {
      uint64_t v = 0;
      for (int k = 0; k < c.widths[w]; k++) {
        int32_t var = c.in_map[off + k];
        uint64_t bitv = model[vb[i] + var - 1] ? 1u : 0u;
        v |= bitv << k;
      }
      words[w] = v;
      off += c.widths[w];
    }
    int r = scuba::verify_words(irs + ir_offsets[i], ir_offsets[i + 1] - ir_offsets[i],
                                words.data(), (int64_t)words.size());
    ok[i] = r == 1 ? 1 : 0;
    if (r != 1) fails.fetch_add(1);
  };
  parallel_for(n, hw_threads(nthreads), [&](int i) {
    try {  // no exception may leave a pool thread
      check(i);
    } catch (...) {
      ok[i] = 0;
      oom.store(true);
    }
  });
  if (oom.load()) {
    scuba::set_error("scuba_verify_batch: out of host memory");
    return SCUBA_ERR_NOMEM;
  }
  return fails.load();
}

}  // extern "C"
