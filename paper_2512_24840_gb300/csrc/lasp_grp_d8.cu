// The grouped tensor-core fit at Legendre degree 8 (its own translation unit).
#include "lasp_grouped.cuh"

namespace lasp {
template int grp_run_deg<8>(Grp&, const TcImages&, const lasp_fit_opts*, cudaStream_t, int*);
}  // namespace lasp
