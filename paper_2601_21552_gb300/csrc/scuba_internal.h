// scuba_internal.h -- declarations shared by the translation units of libscuba.
#pragma once
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>
#include <vector>

namespace scuba {

// A named NVTX range over a scope (encode, upload, prep, search, verify), so a
// profiler's timeline shows where a call spends its time. NVTX is header-only
// and costs next to nothing when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// A CNF in DIMACS numbering (+-v, v in 1..nvars) as produced by the encoder.
struct HostCnf {
  int nvars = 0;
  std::vector<int64_t> clause_begin{0};
  std::vector<int32_t> lits;
  std::vector<int32_t> in_map;  // variable of each input bit, LSB first, FREE order
  std::vector<int32_t> widths;  // width of each FREE word
};

// Bit-blast one serialized query (IR layout in workloads/ir.py). Returns 0 or
// -1 for a malformed IR.
int encode_query(const int64_t* ir, int64_t len, HostCnf* out);

// Evaluate the query's constraints exactly for the given input words.
// Returns 1 (all hold), 0 (some root is false), -1 (malformed IR / bad input).
int verify_words(const int64_t* ir, int64_t len, const uint64_t* words, int64_t nwords);

void set_error(const std::string& msg);

}  // namespace scuba
