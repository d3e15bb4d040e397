// Step kernels with 64-bit population offsets, for grids whose 9 pitch ny
// population slots reach 2^31 (above about 238 million nodes). The same
// templates as the 32-bit kernels of lbm_api.cu, instantiated with
// IX = long long in a translation unit of their own so that the library's
// build stays parallel; the 32-bit instantiations are unchanged.
#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace {

using IX = long long;

template <typename real, int MODE, bool STAGED, bool PADDED>
void *big_ptr(bool walls, bool pres)
{
    using namespace lbm;
    if (walls && pres) return (void *)step_kernel<real, true, true, MODE, STAGED, PADDED, IX>;
    if (walls) return (void *)step_kernel<real, true, false, MODE, STAGED, PADDED, IX>;
    if (pres) return (void *)step_kernel<real, false, true, MODE, STAGED, PADDED, IX>;
    return (void *)step_kernel<real, false, false, MODE, STAGED, PADDED, IX>;
}

template <typename real, int MODE>
void *big_ptr(bool walls, bool pres, bool staged, bool padded)
{
    if (staged)
        return padded ? big_ptr<real, MODE, true, true>(walls, pres) : big_ptr<real, MODE, true, false>(walls, pres);
    return padded ? big_ptr<real, MODE, false, true>(walls, pres) : big_ptr<real, MODE, false, false>(walls, pres);
}

template <bool PADDED>
void *big_rows2_ptr(bool walls, bool pres)
{
    using namespace lbm;
    if (walls && pres) return (void *)step_kernel_rows2<true, true, PADDED, false, IX>;
    if (walls) return (void *)step_kernel_rows2<true, false, PADDED, false, IX>;
    if (pres) return (void *)step_kernel_rows2<false, true, PADDED, false, IX>;
    return (void *)step_kernel_rows2<false, false, PADDED, false, IX>;
}

} // namespace

void *lbm_big_step_kernel_ptr(int precision, int mode, bool walls, bool pres, bool staged, bool padded)
{
    if (precision == 64)
        return mode == lbm::MODE_STEP ? big_ptr<double, lbm::MODE_STEP>(walls, pres, staged, padded)
                                      : big_ptr<double, lbm::MODE_FIELDS>(walls, pres, staged, padded);
    return mode == lbm::MODE_STEP ? big_ptr<float, lbm::MODE_STEP>(walls, pres, staged, padded)
                                  : big_ptr<float, lbm::MODE_FIELDS>(walls, pres, staged, padded);
}

void *lbm_big_rows2_kernel_ptr(bool walls, bool pres, bool padded)
{
    return padded ? big_rows2_ptr<true>(walls, pres) : big_rows2_ptr<false>(walls, pres);
}
