// Type dispatch over the run-time index / value widths.
#pragma once

#include "internal.h"

namespace sp {

template <class F>
sp_status dispatch_i(sp_itype t, F&& f) {
  if (t == SP_I32) return f(int32_t{});
  return f(int64_t{});
}
template <class F>
sp_status dispatch_v(sp_vtype t, F&& f) {
  if (t == SP_F32) return f(uint32_t{});
  return f((unsigned long long){});
}

}  // namespace sp
