// Source-row loaders of the count and fill passes.
//
// A loader describes where listed row i takes its entries from and which survive:
//   struct Loader {
//     using CI = ...;  using VT = ...;           // column index / value word types
//     static constexpr bool kAllKept;            // no source entry is ever dropped
//     static constexpr bool kLoadVals;           // the pass needs the values
//     static constexpr bool kEagerVals;          // load values with the columns, before
//                                                // knowing which survive
//     RowSrc row(int64 i) const;                 // source runs of listed row i
//     const CI* cols(int part) const;            // column / value arrays of run `part`
//     const VT* vals(int part) const;
//     bool test(int part, int64 c) const;        // does an entry of column c survive
//     bool map(int part, int64 c, uint32& key) const;
//         // new column of a surviving entry with column c (false: dropped)
//     static constexpr bool kRowCtx;             // survival depends on the row as well:
//     bool test_ctx(int part, int64 c, int64 i) const;            // instead of test,
//     bool map_ctx(int part, int64 c, uint32& key, int64 i, int64& aux) const;  // map,
//     VT value_ctx(int part, int64 pos, int64 aux) const;          // and the value load
//   };
// Source entries are read in batches (struct Batch): every thread first issues the
// column loads of U entries, then their map lookups, then their value loads, so that
// U independent chains of dependent loads are in flight per thread.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace sp {

struct RowSrc {
  long long s0, s1;  // start of run 0 / run 1 in the source arrays
  long long n0, n1;  // lengths (n1 = 0 for single-run sources)
};

// First position in col[lo, hi) (ascending) whose column is not below v.
template <class CI>
__device__ __forceinline__ long long lower_bound_col(const CI* col, long long lo, long long hi, long long v) {
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if ((long long)col[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// U source entries read together (see the file comment).
template <class Ld, int U>
struct Batch {
  static constexpr int UR = Ld::kRowCtx ? U : 1;
  long long pos[U];
  int part[U];
  bool valid[U];
  bool kept[U];
  uint32_t key[U];
  typename Ld::VT v[U];
  long long row[UR];  // listed row of each entry (row-context loaders only)
  __device__ __forceinline__ void set_row(int u, long long i) {
    if constexpr (Ld::kRowCtx) row[u] = i;
  }
  __device__ __forceinline__ void run(const Ld& ld) {
    using CI = typename Ld::CI;
    CI c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) c[u] = valid[u] ? ld_stream(ld.cols(part[u]) + pos[u]) : CI(0);
    if constexpr (Ld::kRowCtx) {
      long long aux[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        kept[u] = valid[u] && ld.map_ctx(part[u], (long long)c[u], key[u], row[u], aux[u]);
      if constexpr (Ld::kLoadVals) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (kept[u]) v[u] = ld.value_ctx(part[u], pos[u], aux[u]);
      }
    } else {
      if constexpr (Ld::kLoadVals && (Ld::kAllKept || Ld::kEagerVals)) {
        // the value loads need not wait for the map lookups (nothing is dropped, or the
        // loader prefers loading dropped values to another round trip)
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (valid[u]) v[u] = ld_stream(ld.vals(part[u]) + pos[u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) kept[u] = valid[u] && ld.map(part[u], (long long)c[u], key[u]);
      if constexpr (Ld::kLoadVals && !Ld::kAllKept && !Ld::kEagerVals) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (kept[u]) v[u] = ld_stream(ld.vals(part[u]) + pos[u]);
      }
    }
  }
  // entry e of a row's source runs
  __device__ __forceinline__ void at(int u, const RowSrc& rs, long long e) {
    part[u] = e < rs.n0 ? 0 : 1;
    pos[u] = part[u] ? rs.s1 + (e - rs.n0) : rs.s0 + e;
  }
};

constexpr int LOAD_U = 4;  // entries per thread per batch

// A loader whose rows come from arrays recorded by the count pass (source start and
// length of every listed row: one contiguous read instead of the index -> row pointer
// chain), with every survival test and relabel of the underlying single-run loader.
template <class Ld>
struct RecordedRows : Ld {
  const long long* rs0;
  const long long* rsn;
  __device__ __forceinline__ RowSrc row(long long i) const { return RowSrc{rs0[i], 0, rsn[i], 0}; }
};

// A loader view for counting passes: membership only (no key, no value loads).
template <class Ld>
struct CountOnly {
  using CI = typename Ld::CI;
  struct Nothing {};
  using VT = Nothing;
  static constexpr bool kLoadVals = false;
  static constexpr bool kAllKept = false;
  static constexpr bool kEagerVals = false;
  static constexpr bool kRowCtx = Ld::kRowCtx;
  Ld ld;
  __device__ __forceinline__ const CI* cols(int part) const { return ld.cols(part); }
  __device__ __forceinline__ bool map(int part, long long c, uint32_t&) const {
    return ld.test(part, c);
  }
  __device__ __forceinline__ bool map_ctx(int part, long long c, uint32_t&, long long i, long long&) const {
    return ld.test_ctx(part, c, i);
  }
  __device__ __forceinline__ VT value_ctx(int, long long, long long) const { return VT{}; }
};

// Rows whose source holds more than SRC_LONG entries are "source-long": the count and
// fill passes give each of them a whole CTA instead of a warp.
constexpr int SRC_LONG = 1024;

// Whether a row goes to the CTA-per-row kernels by the length of its first run alone (a
// loader declares kLongFirst = true; by default both runs count).
template <class Ld, class = void>
struct long_by_first : std::false_type {};
template <class Ld>
struct long_by_first<Ld, std::void_t<decltype(Ld::kLongFirst)>> : std::bool_constant<Ld::kLongFirst> {};
template <class Ld>
__device__ __forceinline__ bool row_is_long(const RowSrc& rs) {
  return (long_by_first<Ld>::value ? rs.n0 : rs.n0 + rs.n1) > SRC_LONG;
}

}  // namespace sp
