// The state kept between a count call and its fill call (extraction / assignment).
#pragma once

#include "internal.h"

struct sp_plan {
  int op = 0;  // 0 = extraction, 1 = assignment
  sp_csr A{}, B{};
  const void* I = nullptr;
  const void* J = nullptr;
  long long nI = 0, nJ = 0;
  sp_itype idx_type = SP_I32;
  sp_assign_mode mode = SP_ASSIGN_REPLACE;
  long long nnz_out = 0;   // entries of the result
  long long nnz_temp = 0;  // assignment: entries of the rebuilt rows I
  char* buf = nullptr;     // plan-owned device memory
  size_t buf_bytes = 0;
  cudaStream_t stream = nullptr;
  // device pointers inside buf
  void* jmap = nullptr;        // extraction: jinv (nJ positions); assignment: J bitmap
  void* rowmap = nullptr;      // assignment: rowmap (m entries of idx type)
  uint32_t* ibits = nullptr;   // assignment: bitmap of I's rows (m bits)
  void* jbits = nullptr;       // extraction: membership bitmap of J
  void* jinv = nullptr;        // assignment (union modes): column -> position in J
  long long* vp = nullptr;     // extraction: row pointer of B; assignment: of rows I (temp)
  long long* vp_out = nullptr; // assignment: row pointer of A'
  long long* rpB = nullptr;    // assignment: B's row pointer widened to int64
  long long* cl_rows = nullptr;
  // extraction: shape of J (0 general, 1 ascending, 2 consecutive), its first index, and
  // for consecutive J the start of every selected row's kept segment
  int j_shape = 0;  // 3: J repeats indices (multi-map path)
  long long j0 = 0;
  long long* sstart = nullptr;  // consecutive J: kept-segment start; else the source start
  long long* slen = nullptr;    // general J: source length of every listed row
  // repeated J: jcnt[c] = #{b : J[b] = c}, jptr = its exclusive scan, jpos the positions b
  // grouped by column (in the plan's second buffer)
  char* buf2 = nullptr;
  size_t buf2_bytes = 0;
  uint32_t* jcnt = nullptr;
  long long* jptr = nullptr;
  void* jpos = nullptr;
  // extraction, general / ascending J: identify tables (rank map words + member
  // positions, or J sorted with its positions), and the rows the fill queues for sorting
  int identify = 0;
  unsigned long long* jmeta = nullptr;
  void* jrpos = nullptr;
  uint32_t* jsk = nullptr;
  uint32_t* jsp = nullptr;
  long long n_slow = 0;
  long long max_lb = 0;  // assignment: longest row of B (the merge fill takes rows of at most 32)
  long long list_cap = 0;
  unsigned* counters = nullptr;  // [0] n_cl [3] count ticket [4] rows of more than XFAST entries
  long long* h_tail = nullptr;   // the context's pinned scratch: totals read back by the count call
};

namespace sp {
sp_status store_rowptr(sp_ctx* ctx, cudaStream_t s, const long long* vp, long long n1, sp_itype t,
                       void* out);
sp_status widen_rowptr(sp_ctx* ctx, cudaStream_t s, const void* in, sp_itype t, long long n1,
                       long long* out);
sp_status plan_alloc(sp_ctx* ctx, sp_plan* pl, size_t bytes, cudaStream_t s);
sp_status plan_release(sp_ctx* ctx, sp_plan* pl);
}  // namespace sp
