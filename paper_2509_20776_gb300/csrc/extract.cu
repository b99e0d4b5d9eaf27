// sp_extract: B = A(I, J), B[i, j] = A[I[i], J[j]]  (Sec. 2.2; HipExtract, Algorithms 3, 5).
//
// Identify: the columns of J become a rank map (membership bit + rank per column and the
// position of every member: the SpQvec_inv of Algorithm 3 in compact form) or J sorted
// once (Algorithm 5's binary search); the first pass of Algorithm 5 counts the entries
// of each selected row that survive (a warp ballot + popc per 32 entries); the
// exclusive scan of the counts is B's row pointer.  Fill: the surviving entries are
// relabelled and sorted per row and written once at their final place (Algorithm 5's
// second pass and the Build step; extract_rows.cuh).  Rows of I may repeat; J with
// repeats takes the multi-map path below.
#include "dispatch.h"
#include "extract_rows.cuh"
#include "kernels.cuh"
#include "plan.h"
#include "rowsort.cuh"

namespace sp {

// Consecutive J = [j0, j1): the kept entries of a (sorted) row form one segment, found by
// binary search, and keep their order (the paper's binary-search idea of Alg. 5 applied
// to a whole range).  The row length functor of the scan records the segment start.
template <class RP, class CI, class IX>
struct ExtractRangeLen {
  const RP* rowptr;
  const CI* col;
  const IX* I;
  long long m, nnz, j0, j1;
  long long* sstart;
  DevStatus* st;
  __device__ long long operator()(long long i) const {
    const long long r = (long long)I[i];
    long long s = 0, e = 0;
    if (r < 0 || r >= m) {
      dev_fail(st, SP_ERR_INDEX_RANGE, i);
    } else {
      s = (long long)rowptr[r];
      e = (long long)rowptr[r + 1];
      if (s < 0 || e < s || e > nnz) s = e = 0;
    }
    const long long lo = lower_bound_col(col, s, e, j0), hi = lower_bound_col(col, lo, e, j1);
    sstart[i] = lo;
    return hi - lo;
  }
};

template <class CIt, class VTt>
struct ExtractRangeGs {
  using CI = CIt;
  using VT = VTt;
  const CI* c_;
  const VT* v_;
  const long long* sstart;
  long long j0;
  __device__ long long src(long long i) const { return sstart[i]; }
  __device__ CI col(long long pos) const { return ld_stream(c_ + pos); }
  __device__ VT val(long long pos) const { return ld_stream(v_ + pos); }
  __device__ CI map(long long, CI c) const { return CI((long long)c - j0); }
};

// Repeated J (Sec. 2.2 allows repeats): column c of A feeds every position b with
// J[b] = c.  The map is a CSR of the inverse: jcnt[c] positions starting at jptr[c] in
// jpos.  One warp per listed row counts (pass 0: sum of jcnt over the row's columns)
// or fills (pass 1: an entry with column c writes its value under each of its
// positions, slots from a warp scan of the multiplicities); the row sort orders them.
template <class IX>
__global__ void k_jmulti_count(const IX* __restrict__ J, long long nJ, long long n, uint32_t* jcnt) {
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nJ;
       b += (long long)gridDim.x * blockDim.x) {
    const long long c = (long long)J[b];
    if (c >= 0 && c < n) atomicAdd(jcnt + c, 1u);  // out-of-range J was reported
  }
}

template <class IX>
__global__ void k_jmulti_fill(const IX* __restrict__ J, long long nJ, long long n,
                              const long long* __restrict__ jptr, uint32_t* jfill, IX* __restrict__ jpos) {
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nJ;
       b += (long long)gridDim.x * blockDim.x) {
    const long long c = (long long)J[b];
    if (c < 0 || c >= n) continue;
    jpos[jptr[c] + atomicAdd(jfill + c, 1u)] = IX(b);
  }
}

template <int PASS, class RP, class CI, class VT, class IX>
__global__ void k_extract_multi(const RP* __restrict__ rowptr, const CI* __restrict__ col,
                                const VT* __restrict__ val, const IX* __restrict__ I, long long nI,
                                long long m, long long n, long long nnz, const uint32_t* __restrict__ jcnt,
                                const long long* __restrict__ jptr, const IX* __restrict__ jpos,
                                long long* __restrict__ vp, CI* __restrict__ out_col,
                                VT* __restrict__ out_val, DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = w0; i < nI; i += nw) {
    const long long r = (long long)I[i];
    long long s = 0, e = 0;
    if (r >= 0 && r < m) {
      s = (long long)rowptr[r];
      e = (long long)rowptr[r + 1];
      if (s < 0 || e < s || e > nnz) s = e = 0;
    }
    long long run = PASS ? vp[i] : 0;
    const long long end = PASS ? vp[i + 1] : 0;
    for (long long k0 = s; k0 < e; k0 += 32) {
      const long long k = k0 + lane;
      long long c = -1;
      long long mlt = 0;
      if (k < e) {
        c = (long long)ld_stream(col + k);
        if (c >= 0 && c < n) mlt = jcnt[c];
      }
      if (PASS == 0) {
        run += warp_sum(mlt);
      } else {
        const long long incl = warp_incl_sum(mlt);
        const long long base = run + incl - mlt;
        if (mlt) {
          const VT v = ld_stream(val + k);
          const long long p0 = jptr[c];
          for (long long t = 0; t < mlt; ++t) {
            if (base + t < end) {
              st_stream(out_col + base + t, CI(jpos[p0 + t]));
              st_stream(out_val + base + t, v);
            } else {
              dev_fail(st, SP_ERR_INTERNAL, -24);
            }
          }
        }
        run += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    if (PASS == 0 && lane == 0) vp[i] = run;
  }
}

// copy an int64 row pointer into a typed output row pointer
sp_status store_rowptr(sp_ctx* ctx, cudaStream_t s, const long long* vp, long long n1,
                       sp_itype t, void* out) {
  if (t == SP_I64) {
    if ((void*)vp != out) SP_CUDA(cudaMemcpyAsync(out, vp, size_t(n1) * 8, cudaMemcpyDeviceToDevice, s));
    return SP_OK;
  }
  {
    SP_PHASE(SP_PHASE_OTHER);
    k_narrow<int32_t><<<grid_for(n1, 256, ctx->num_sms * 8), 256, 0, s>>>(vp, n1, static_cast<int32_t*>(out),
                                                                         ctx->dstatus);
  }
  SP_CUDA(cudaGetLastError());
  return SP_OK;
}

sp_status widen_rowptr(sp_ctx* ctx, cudaStream_t s, const void* in, sp_itype t, long long n1,
                       long long* out) {
  if (t == SP_I64) {
    SP_CUDA(cudaMemcpyAsync(out, in, size_t(n1) * 8, cudaMemcpyDeviceToDevice, s));
    return SP_OK;
  }
  {
    SP_PHASE(SP_PHASE_OTHER);
    k_widen<int32_t><<<grid_for(n1, 256, ctx->num_sms * 8), 256, 0, s>>>(static_cast<const int32_t*>(in), n1, out);
  }
  SP_CUDA(cudaGetLastError());
  return SP_OK;
}

sp_status plan_alloc(sp_ctx* ctx, sp_plan* pl, size_t bytes, cudaStream_t s) {
  pl->buf = static_cast<char*>(ctx_alloc(ctx, bytes, s));
  if (!pl->buf) return SP_ERR_OOM;
  pl->buf_bytes = bytes;
  pl->h_tail = ctx->hbuf;  // every use is read back before the count call returns
  return SP_OK;
}

template <class RP, class CI, class IX>
sp_status extract_count_impl(sp_ctx* ctx, sp_plan* pl, cudaStream_t s) {
  const sp_csr& A = pl->A;
  const long long m = A.nrows, n = A.ncols, nnz = A.nnz, nI = pl->nI, nJ = pl->nJ;
  const IX* I = static_cast<const IX*>(pl->I);
  const IX* J = static_cast<const IX*>(pl->J);
  pl->identify = ctx->cur.identify;
  const long long nw32 = (n + 31) / 32;
  Carver cv;
  const size_t o_meta = cv.reserve(pl->identify == 0 ? size_t(nw32) * 8 : 0);
  const size_t o_jrp = cv.reserve(pl->identify == 0 ? size_t(nJ) * sizeof(IX) : 0);
  const size_t o_jsk = cv.reserve(pl->identify == 1 ? size_t(nJ) * 4 : 0);
  const size_t o_jsp = cv.reserve(pl->identify == 1 ? size_t(nJ) * 4 : 0);
  const size_t o_vp2 = cv.reserve(16);
  const size_t o_jb = cv.reserve(size_t(nw32) * 4);
  const size_t o_vp = cv.reserve(size_t(nI + 1) * 8);
  pl->list_cap = nI + 1;
  const size_t o_cl = cv.reserve(size_t(pl->list_cap) * 8);
  const size_t o_cn = cv.reserve(64);
  const size_t o_scan = cv.reserve(scan_ws_bytes(nI > nw32 ? nI : nw32));
  const size_t o_ss = cv.reserve(size_t(nI) * 8);
  const size_t o_sn = cv.reserve(size_t(nI) * 8);
  const size_t o_fl = cv.reserve(16);  // J strictly ascending / consecutive / repeats
  SP_TRY(plan_alloc(ctx, pl, cv.total(), s));
  cv.bind(pl->buf);
  pl->sstart = cv.at<long long>(o_ss);
  pl->slen = cv.at<long long>(o_sn);
  pl->jmeta = cv.at<unsigned long long>(o_meta);
  pl->jrpos = cv.at<void>(o_jrp);
  pl->jsk = cv.at<uint32_t>(o_jsk);
  pl->jsp = cv.at<uint32_t>(o_jsp);
  uint32_t* jbits = cv.at<uint32_t>(o_jb);
  pl->jbits = jbits;
  pl->vp = cv.at<long long>(o_vp);
  pl->cl_rows = cv.at<long long>(o_cl);
  pl->counters = cv.at<unsigned>(o_cn);
  const int nsm = ctx->num_sms;
  // the shape of J picks the path: consecutive J needs neither maps nor membership tests
  int* flags = cv.at<int>(o_fl);
  SP_CUDA(cudaMemsetAsync(flags, 0, 16, s));
  if (nJ > 1) {
    {
      SP_PHASE(SP_PHASE_MAP);
      k_index_shape<IX><<<grid_for(nJ, 256, nsm * 8), 256, 0, s>>>(J, nJ, flags);
    }
    SP_CUDA(cudaGetLastError());
  }
  // membership bitmap of J; repeats are flagged (flags[2]) and take the multi-map path
  SP_CUDA(cudaMemsetAsync(jbits, 0, size_t((n + 31) / 32) * 4, s));
  if (nJ > 0) {
    {
      SP_PHASE(SP_PHASE_MAP);
      k_mark_bits<IX><<<grid_for(nJ, 256, nsm * 8), 256, 0, s>>>(J, nJ, n, jbits, ctx->dstatus,
                                                                  SP_ERR_DUPLICATE_INDEX, flags + 2);
    }
    SP_CUDA(cudaGetLastError());
  }
  SP_CUDA(cudaMemcpyAsync(pl->h_tail + 1, flags, 16, cudaMemcpyDeviceToHost, s));
  if (nJ > 0) SP_CUDA(cudaMemcpyAsync(pl->h_tail + 3, J, sizeof(IX), cudaMemcpyDeviceToHost, s));
  SP_TRY(ctx_collect(ctx, s));
  int fl[3];
  std::memcpy(fl, pl->h_tail + 1, 12);
  pl->j_shape = nJ == 0 ? 0 : (fl[2] ? 3 : (fl[1] == 0 ? 2 : (fl[0] == 0 ? 1 : 0)));
  if (pl->j_shape == 3) {
    if (nI > 0) {
      SP_PHASE(SP_PHASE_MAP);
      k_range_check<IX><<<grid_for(nI, 256, nsm * 8), 256, 0, s>>>(I, nI, m, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
    Carver c2;
    const size_t o_cnt = c2.reserve(size_t(n) * 4);
    const size_t o_fil = c2.reserve(size_t(n) * 4);
    const size_t o_ptr = c2.reserve(size_t(n + 1) * 8);
    const size_t o_pos = c2.reserve(size_t(nJ) * sizeof(IX));
    const size_t o_sc2 = c2.reserve(scan_ws_bytes(n));
    pl->buf2 = static_cast<char*>(ctx_alloc(ctx, c2.total(), s));
    if (!pl->buf2) return SP_ERR_OOM;
    pl->buf2_bytes = c2.total();
    c2.bind(pl->buf2);
    pl->jcnt = c2.at<uint32_t>(o_cnt);
    uint32_t* jfill = c2.at<uint32_t>(o_fil);
    pl->jptr = c2.at<long long>(o_ptr);
    IX* jpos = c2.at<IX>(o_pos);
    pl->jpos = jpos;
    SP_CUDA(cudaMemsetAsync(pl->jcnt, 0, size_t(n) * 4, s));
    SP_CUDA(cudaMemsetAsync(jfill, 0, size_t(n) * 4, s));
    {
      SP_PHASE(SP_PHASE_MAP);
      k_jmulti_count<IX><<<grid_for(nJ, 256, nsm * 8), 256, 0, s>>>(J, nJ, n, pl->jcnt);
    }
    SP_CUDA(cudaGetLastError());
    SP_TRY(launch_scan(ctx, s, LoadArray<uint32_t>{pl->jcnt},
                       StoreDual<long long>{pl->jptr, nullptr, ctx->dstatus}, n, c2.at<char>(o_sc2)));
    {
      SP_PHASE(SP_PHASE_MAP);
      k_jmulti_fill<IX><<<grid_for(nJ, 256, nsm * 8), 256, 0, s>>>(J, nJ, n, pl->jptr, jfill, jpos);
    }
    SP_CUDA(cudaGetLastError());
    if (nI > 0) {
      SP_PHASE(SP_PHASE_COUNT);
      k_extract_multi<0, RP, CI, uint32_t, IX><<<grid_for(nI * 32, 256, nsm * 16), 256, 0, s>>>(
          static_cast<const RP*>(A.rowptr), static_cast<const CI*>(A.colidx), nullptr, I, nI, m, n, nnz,
          pl->jcnt, pl->jptr, jpos, pl->vp, nullptr, nullptr, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
    SP_TRY(launch_scan(ctx, s, LoadArray<long long>{pl->vp},
                       StoreDual<long long>{pl->vp, nullptr, ctx->dstatus}, nI, cv.at<char>(o_scan)));
    SP_CUDA(cudaMemcpyAsync(pl->h_tail, pl->vp + nI, 8, cudaMemcpyDeviceToHost, s));
    SP_TRY(ctx_collect(ctx, s));
    pl->nnz_out = pl->h_tail[0];
    return SP_OK;
  }
  if (pl->j_shape == 2) {
    IX first;
    std::memcpy(&first, pl->h_tail + 3, sizeof(IX));
    pl->j0 = (long long)first;
    if (pl->j0 < 0 || pl->j0 + nJ > n) return SP_ERR_INDEX_RANGE;
    ExtractRangeLen<RP, CI, IX> len{static_cast<const RP*>(A.rowptr), static_cast<const CI*>(A.colidx), I,
                                    m, nnz, pl->j0, pl->j0 + nJ, pl->sstart, ctx->dstatus};
    SP_TRY(launch_scan(ctx, s, len, StoreDual<long long>{pl->vp, nullptr, ctx->dstatus}, nI,
                       cv.at<char>(o_scan)));
    SP_CUDA(cudaMemcpyAsync(pl->h_tail, pl->vp + nI, 8, cudaMemcpyDeviceToHost, s));
    SP_TRY(ctx_collect(ctx, s));
    pl->nnz_out = pl->h_tail[0];
    return SP_OK;
  }
  // general or ascending J: identify tables, then the count
  SP_CUDA(cudaMemsetAsync(pl->counters, 0, 64, s));
  if (pl->identify == 0) {
    if (nJ > 0) {
      // rank words: bits | exclusive prefix of the words' popcounts; then the positions
      SP_TRY(launch_scan(ctx, s, LoadPopc{jbits}, StoreRank{jbits, pl->jmeta, nw32}, nw32, cv.at<char>(o_scan),
                         SP_PHASE_MAP));
      {
        SP_PHASE(SP_PHASE_MAP);
        k_jrank_pos<IX><<<grid_for(nJ, 256, nsm * 8), 256, 0, s>>>(J, nJ, n, pl->jmeta, static_cast<IX*>(pl->jrpos));
      }
      SP_CUDA(cudaGetLastError());
    }
  } else if (nJ > 0) {
    // J sorted once, its positions carried as values (one row of nJ keys)
    {
      SP_PHASE(SP_PHASE_MAP);
      k_jsorted_init<IX><<<grid_for(nJ, 256, nsm * 8), 256, 0, s>>>(J, nJ, pl->jsk, pl->jsp);
    }
    SP_CUDA(cudaGetLastError());
    long long* vp2 = cv.at<long long>(o_vp2);
    pl->h_tail[4] = 0;
    pl->h_tail[5] = nJ;
    SP_CUDA(cudaMemcpyAsync(vp2, pl->h_tail + 4, 16, cudaMemcpyHostToDevice, s));
    Carver cw;
    size_t ro[kRowsSlots];
    rows_reserve(cw, 1, nJ, 4, ro);
    char* base;
    SP_TRY(ctx_workspace(ctx, cw.total(), s, &base));
    cw.bind(base);
    const RowsWs w = rows_bind(cw, 1, nJ, ro);
    SP_TRY((run_rows<uint32_t, uint32_t, NoGather<uint32_t, uint32_t>>(ctx, s, vp2, 1, nJ, ceil_log2_u64(uint64_t(n)),
                                                                       w, nullptr, true, pl->jsk, pl->jsp)));
  }
  if (nI > 0) {
    const RP* rp = static_cast<const RP*>(A.rowptr);
    const CI* ci = static_cast<const CI*>(A.colidx);
    const long long groups = (nI + 31) / 32;
    const int g = grid_for(groups * 32, XB, nsm * 8);
    CountLists cl{pl->cl_rows, pl->counters + 0, pl->list_cap};
    auto count = [&](auto test) -> sp_status {
      using Test = decltype(test);
      {
        SP_PHASE(SP_PHASE_COUNT);
        const XOne<CI, uint32_t, Test> src{ci, nullptr, test};
        const XResolveI<RP, IX> res{rp, I, m, nnz, pl->sstart, pl->slen, ctx->dstatus};
        k_xcount<<<g, XB, 0, s>>>(src, res, nI, pl->vp, pl->cl_rows, pl->counters + 0, pl->list_cap, pl->counters + 4,
                                  ctx->dstatus);
      }
      SP_CUDA(cudaGetLastError());
      const XLongRows<CI, uint32_t, Test> lr{ci, nullptr, test, pl->sstart, pl->slen};
      {
        SP_PHASE(SP_PHASE_COUNT);
        k_count_long<<<nsm, 1024, 0, s>>>(lr, pl->vp, cl, pl->counters + 3, ctx->dstatus);
      }
      SP_CUDA(cudaGetLastError());
      return SP_OK;
    };
    if (pl->identify == 0) SP_TRY(count(JBits{jbits, n}));
    else SP_TRY(count(JSorted{pl->jsk, pl->jsp, nJ}));
  }
  SP_TRY(launch_scan(ctx, s, LoadArray<long long>{pl->vp},
                     StoreDual<long long>{pl->vp, nullptr, ctx->dstatus}, nI, cv.at<char>(o_scan)));
  SP_CUDA(cudaMemcpyAsync(pl->h_tail, pl->vp + nI, 8, cudaMemcpyDeviceToHost, s));
  SP_CUDA(cudaMemcpyAsync(pl->h_tail + 6, pl->counters + 4, 4, cudaMemcpyDeviceToHost, s));
  SP_TRY(ctx_collect(ctx, s));
  pl->nnz_out = pl->h_tail[0];
  pl->n_slow = (long long)*reinterpret_cast<const unsigned*>(pl->h_tail + 6);
  return SP_OK;
}

template <class RP, class CI, class VT, class IX>
sp_status extract_fill_impl(sp_ctx* ctx, sp_plan* pl, sp_csr* B, cudaStream_t s) {
  const sp_csr& A = pl->A;
  const long long nI = pl->nI, nnz_out = pl->nnz_out;
  SP_TRY(store_rowptr(ctx, s, pl->vp, nI + 1, B->rowptr_type, B->rowptr));
  if (nnz_out == 0) return SP_OK;
  CI* oc = static_cast<CI*>(B->colidx);
  VT* ov = static_cast<VT*>(B->values);
  Carver cv;
  size_t ro[kRowsSlots];
  if (pl->j_shape == 2) {
    // consecutive J: copy every row's kept segment, columns shifted by j0; already sorted
    rows_reserve(cv, nI, nnz_out, sizeof(VT), ro, false);
    char* base;
    SP_TRY(ctx_workspace(ctx, cv.total(), s, &base));
    cv.bind(base);
    const ExtractRangeGs<CI, VT> g{static_cast<const CI*>(A.colidx), static_cast<const VT*>(A.values),
                                   pl->sstart, pl->j0};
    const RowsWs w = rows_bind(cv, nI, nnz_out, ro, false);
    return run_rows(ctx, s, pl->vp, nI, nnz_out, 0, w, &g, false, oc, ov);
  }
  if (pl->j_shape == 3) {
    // repeated J: every kept entry once per position of its column, then the row sort
    rows_reserve(cv, nI, nnz_out, sizeof(VT), ro);
    char* base;
    SP_TRY(ctx_workspace(ctx, cv.total(), s, &base));
    cv.bind(base);
    {
      SP_PHASE(SP_PHASE_GATHER);
      k_extract_multi<1, RP, CI, VT, IX><<<grid_for(nI * 32, 256, ctx->num_sms * 16), 256, 0, s>>>(
          static_cast<const RP*>(A.rowptr), static_cast<const CI*>(A.colidx), static_cast<const VT*>(A.values),
          static_cast<const IX*>(pl->I), nI, A.nrows, A.ncols, A.nnz, pl->jcnt, pl->jptr,
          static_cast<const IX*>(pl->jpos), pl->vp, oc, ov, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
    const RowsWs w = rows_bind(cv, nI, nnz_out, ro);
    const int kb = ceil_log2_u64(uint64_t(pl->nJ));
    return run_rows<CI, VT, NoGather<CI, VT>>(ctx, s, pl->vp, nI, nnz_out, kb, w, nullptr, true, oc, ov);
  }
  const bool sorted = pl->j_shape == 1;  // ascending J: the relabelling keeps rows in order
  rows_reserve(cv, nI, nnz_out, sizeof(VT), ro, !sorted, pl->n_slow);
  const size_t o_tk = cv.reserve(16);
  char* base;
  SP_TRY(ctx_workspace(ctx, cv.total(), s, &base));
  cv.bind(base);
  const RowsWs w = rows_bind(cv, nI, nnz_out, ro, !sorted, pl->n_slow);
  unsigned* ticket = cv.at<unsigned>(o_tk);
  SP_CUDA(cudaMemsetAsync(ticket, 0, 16, s));
  SP_CUDA(cudaMemsetAsync(w.counters, 0, 16 * 4, s));
  const int nsm = ctx->num_sms;
  const int kb = ceil_log2_u64(uint64_t(pl->nJ));
  const CI* ci = static_cast<const CI*>(A.colidx);
  const VT* vv = static_cast<const VT*>(A.values);
  const long long groups = (nI + 31) / 32;
  const int g = grid_for(groups * 32, XB, nsm * 8);
  const int lane_rows = pl->nJ <= 0xFFFFFFFFll ? XF_LANE : 0;  // keys (positions in J) below the padding key
  auto fill = [&](auto rel) -> sp_status {
    using Rel = decltype(rel);
    {
      SP_PHASE(SP_PHASE_GATHER);
      const XOne<CI, VT, Rel> src{ci, vv, rel};
      if (sorted)
        k_xfill<XOne<CI, VT, Rel>, true><<<g, XB, 0, s>>>(src, nI, pl->sstart, pl->slen, pl->vp, oc, ov, w.fin,
                                                          w.counters + 0, w.fin_cap, w.huge, w.huge_n(),
                                                          w.huge_cap, kb, lane_rows, ctx->dstatus);
      else
        k_xfill<XOne<CI, VT, Rel>, false><<<g, XB, 0, s>>>(src, nI, pl->sstart, pl->slen, pl->vp, oc, ov, w.fin,
                                                           w.counters + 0, w.fin_cap, w.huge, w.huge_n(),
                                                           w.huge_cap, kb, lane_rows, ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
    // rows of more than SRC_LONG source entries: one CTA each, kept entries in source order
    const XLongRows<CI, VT, Rel> lr{ci, vv, rel, pl->sstart, pl->slen};
    {
      SP_PHASE(SP_PHASE_GATHER);
      k_fill_long<<<nsm, 1024, 0, s>>>(lr, pl->cl_rows, pl->counters + 0, pl->list_cap, pl->vp, ticket, oc, ov,
                                       ctx->dstatus);
    }
    SP_CUDA(cudaGetLastError());
    return SP_OK;
  };
  if (pl->identify == 0)
    SP_TRY(fill(JRank<IX>{pl->jmeta, static_cast<const IX*>(pl->jrpos), A.ncols}));
  else
    SP_TRY(fill(JSorted{pl->jsk, pl->jsp, pl->nJ}));
  if (sorted) return SP_OK;
  // the rows the warp path did not sort (more than XFAST source entries)
  return sort_queued<CI, VT>(ctx, s, w, kb, oc, ov);
}

sp_status plan_release(sp_ctx* ctx, sp_plan* pl) {
  if (!pl) return SP_OK;
  if (pl->buf) ctx_free(ctx, pl->buf, pl->buf_bytes, pl->stream);
  if (pl->buf2) ctx_free(ctx, pl->buf2, pl->buf2_bytes, pl->stream);
  delete pl;
  return SP_OK;
}

}  // namespace sp

using namespace sp;

static sp_status check_index_args(const sp_csr* A, const void* I, long long nI, const void* J,
                                  long long nJ, sp_itype idx_type) {
  if (idx_type != SP_I32 && idx_type != SP_I64) return SP_ERR_INVALID_ARG;
  if (nI < 0 || nJ < 0) return SP_ERR_SHAPE;
  if ((nI > 0 && !I) || (nJ > 0 && !J)) return SP_ERR_INVALID_ARG;
  if (idx_type == SP_I32 && (A->nrows > INT32_MAX || A->ncols > INT32_MAX || nI > INT32_MAX ||
                             nJ > INT32_MAX))
    return SP_ERR_OVERFLOW;
  return SP_OK;
}

extern "C" sp_status sp_extract_count(sp_ctx* ctx, const sp_csr* A, const void* I, int64_t nI,
                                      const void* J, int64_t nJ, sp_itype idx_type,
                                      sp_plan** plan, int64_t* nnz_out, sp_stream_t stream) {
  if (!ctx || !A || !plan || !nnz_out) return SP_ERR_INVALID_ARG;
  *plan = nullptr;
  SP_TRY(check_csr(A));
  SP_TRY(check_index_args(A, I, nI, J, nJ, idx_type));
  if (nJ > J_KEY_LIMIT) return SP_ERR_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  SP_CUDA(cudaSetDevice(ctx->device));
  ctx_begin_call(ctx, SP_OP_EXTRACT, A->nnz);
  SP_TRY(validate_if_asked(ctx, A, s));
  sp_plan* pl = new sp_plan();
  pl->op = 0;
  pl->A = *A;
  pl->I = I;
  pl->J = J;
  pl->nI = nI;
  pl->nJ = nJ;
  pl->idx_type = idx_type;
  pl->stream = s;
  sp_status st = dispatch_i(A->rowptr_type, [&](auto rp) {
    using RP = decltype(rp);
    return dispatch_i(A->colidx_type, [&](auto ci) {
      using CI = decltype(ci);
      return dispatch_i(idx_type, [&](auto ix) {
        using IX = decltype(ix);
        return extract_count_impl<RP, CI, IX>(ctx, pl, s);
      });
    });
  });
  if (st != SP_OK) {
    plan_release(ctx, pl);
    return st;
  }
  *plan = pl;
  *nnz_out = pl->nnz_out;
  return SP_OK;
}

extern "C" sp_status sp_extract_fill(sp_ctx* ctx, sp_plan* pl, sp_csr* B, sp_stream_t stream) {
  if (!ctx || !pl || !B || pl->op != 0) return SP_ERR_INVALID_ARG;
  if (B->rowptr_type != SP_I32 && B->rowptr_type != SP_I64) return SP_ERR_INVALID_ARG;
  if (B->rowptr_type == SP_I32 && pl->nnz_out > INT32_MAX) return SP_ERR_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  SP_CUDA(cudaSetDevice(ctx->device));
  ctx_begin_call(ctx, SP_OP_EXTRACT, pl->A.nnz);
  pl->stream = s;
  B->nrows = pl->nI;
  B->ncols = pl->nJ;
  B->nnz = pl->nnz_out;
  B->colidx_type = pl->A.colidx_type;
  B->value_type = pl->A.value_type;
  const bool owned = lib_allocates(B);
  SP_TRY(alloc_csr(ctx, B, s));
  const sp_csr& A = pl->A;
  const sp_status st_ = dispatch_i(A.rowptr_type, [&](auto rp) {
    using RP = decltype(rp);
    return dispatch_i(A.colidx_type, [&](auto ci) {
      using CI = decltype(ci);
      return dispatch_v(A.value_type, [&](auto vt) {
        using VT = decltype(vt);
        return dispatch_i(pl->idx_type, [&](auto ix) {
          using IX = decltype(ix);
          return extract_fill_impl<RP, CI, VT, IX>(ctx, pl, B, s);
        });
      });
    });
  });
  return release_on_error(ctx, B, owned, s, st_);
}

extern "C" sp_status sp_extract(sp_ctx* ctx, const sp_csr* A, const void* I, int64_t nI,
                                const void* J, int64_t nJ, sp_itype idx_type, sp_csr* B,
                                sp_stream_t stream) {
  if (!B) return SP_ERR_INVALID_ARG;
  sp_plan* pl = nullptr;
  int64_t nnz = 0;
  SP_TRY(sp_extract_count(ctx, A, I, nI, J, nJ, idx_type, &pl, &nnz, stream));
  sp_status st = sp_extract_fill(ctx, pl, B, stream);
  plan_release(ctx, pl);
  return st;
}

extern "C" sp_status sp_kept_counts(sp_ctx* ctx, const sp_csr* A, const void* I, int64_t nI,
                                    const void* J, int64_t nJ, sp_itype idx_type,
                                    int64_t* counts, sp_stream_t stream) {
  if (!ctx || !A || (nI > 0 && !counts)) return SP_ERR_INVALID_ARG;
  sp_plan* pl = nullptr;
  int64_t nnz = 0;
  SP_TRY(sp_extract_count(ctx, A, I, nI, J, nJ, idx_type, &pl, &nnz, stream));
  cudaStream_t s = (cudaStream_t)stream;
  // counts[i] = vp[i+1] - vp[i]
  sp_status st = SP_OK;
  if (nI > 0) {
    {
      SP_PHASE(SP_PHASE_COUNT);
      k_diff<0><<<grid_for(nI, 256, ctx->num_sms * 8), 256, 0, s>>>(pl->vp, nI, reinterpret_cast<long long*>(counts));
    }
    if (cudaGetLastError() != cudaSuccess) st = SP_ERR_CUDA;
  }
  plan_release(ctx, pl);
  return st;
}

extern "C" sp_status sp_plan_destroy(sp_ctx* ctx, sp_plan* plan) {
  if (!plan) return SP_OK;
  if (!ctx) return SP_ERR_INVALID_ARG;
  return plan_release(ctx, plan);
}
