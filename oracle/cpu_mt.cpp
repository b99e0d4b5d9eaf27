// Multithreaded CPU permutation B = P A Q^T (arXiv 2509.20776, Sec. 2.1 and Algorithm 2's
// local computation), the host-core baseline of the measurements.
//
// TEST AND MEASUREMENT INFRASTRUCTURE ONLY: called by the bench's CPU-baseline leg and by
// tests; never by the library, with which it shares no code.
//
// Algorithm 2 computes a process's local piece in two passes over its rows: a count pass
// sizes the output of every destination, a prefix sum turns the counts into offsets, and a
// fill pass writes every entry at its place; the Build step then sorts the received
// entries.  On one shared-memory host the destinations are the output rows themselves:
//   count   len(B[i, :]) = len(A[p[i], :])                 (parallel over rows)
//   scan    B.rowptr = exclusive prefix sum of the lengths  (per-thread blocks, then a
//           scan of the block sums)
//   fill    B.col[k] = qinv[A.col[k']], B.val[k] = A.val[k'] for the entries of row p[i]
//   sort    each row by its new column                      (parallel over rows)
// with qinv[q[j]] = j (the index/value swap of the Identify step).  Values move as 32-bit
// words; rows are sorted as packed (column, value) 64-bit keys.
#include <omp.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

extern "C" {

int sp_cpu_threads(void) { return omp_get_max_threads(); }

// rowptr: m+1, col / val: nnz, p: m (new row -> old row), q: n (new column -> old column)
// or NULL for q = p (square A).  Outputs: out_rowptr m+1, out_col / out_val nnz.
// Returns 0, or -1 when p or q is not a permutation.
int sp_cpu_permute(int64_t m, int64_t n, const int64_t* rowptr, const int32_t* col, const uint32_t* val,
                   const int64_t* p, const int64_t* q, int64_t* out_rowptr, int32_t* out_col, uint32_t* out_val) {
  if (!q) q = p;
  std::vector<int32_t> qinv(size_t(n), -1);
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t j = 0; j < n; ++j) {
    const int64_t c = q[j];
    if (c < 0 || c >= n) bad = 1;
    else qinv[size_t(c)] = int32_t(j);
  }
  if (bad) return -1;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t j = 0; j < n; ++j) bad |= qinv[size_t(j)] < 0;
  if (bad) return -1;
  // count pass: the output length of every row
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t i = 0; i < m; ++i) {
    const int64_t r = p[i];
    if (r < 0 || r >= m) {
      bad = 1;
      out_rowptr[i + 1] = 0;
    } else {
      out_rowptr[i + 1] = rowptr[r + 1] - rowptr[r];
    }
  }
  if (bad) return -1;
  // exclusive scan: per-thread block sums, a scan of those, then the blocks
  const int T = omp_get_max_threads();
  std::vector<int64_t> part(size_t(T) + 1, 0);
  out_rowptr[0] = 0;
#pragma omp parallel num_threads(T)
  {
    const int t = omp_get_thread_num(), nt = omp_get_num_threads();
    const int64_t a = m * t / nt, b = m * (t + 1) / nt;
    int64_t s = 0;
    for (int64_t i = a; i < b; ++i) s += out_rowptr[i + 1];
    part[size_t(t) + 1] = s;
#pragma omp barrier
#pragma omp single
    for (int k = 1; k <= nt; ++k) part[size_t(k)] += part[size_t(k) - 1];
    int64_t run = part[size_t(t)];
    for (int64_t i = a; i < b; ++i) {
      run += out_rowptr[i + 1];
      out_rowptr[i + 1] = run;
    }
  }
  // fill pass and the per-row sort (rows of very different lengths: dynamic schedule)
#pragma omp parallel
  {
    std::vector<uint64_t> buf;
#pragma omp for schedule(dynamic, 256)
    for (int64_t i = 0; i < m; ++i) {
      const int64_t r = p[i], s = rowptr[r], L = rowptr[r + 1] - s, o = out_rowptr[i];
      buf.resize(size_t(L));
      for (int64_t k = 0; k < L; ++k)
        buf[size_t(k)] = (uint64_t(uint32_t(qinv[size_t(col[s + k])])) << 32) | val[s + k];
      std::sort(buf.begin(), buf.end());
      for (int64_t k = 0; k < L; ++k) {
        out_col[o + k] = int32_t(buf[size_t(k)] >> 32);
        out_val[o + k] = uint32_t(buf[size_t(k)]);
      }
    }
  }
  return 0;
}

}  // extern "C"
