// The two-pixels-per-thread instantiations of the compositing backward
// (gs_raster_bwd.cuh), fp32: a translation unit of their own so that they
// compile in parallel with gs_raster.cu.
#include "gs_raster_bwd.cuh"

namespace gs {

RasterBwdKernel<float> raster_bwd_px2_kernel(bool cull, bool atomic, bool persistent, bool any_c, int batch)
{
#define GS_BWD2(CULL, AT, PE, AC, B) k_raster_bwd<float, CULL, AT, PE, AC, 2, B>
    if (batch == 64) {
        static const RasterBwdKernel<float> t[2][2][2][2] = {
            {{{GS_BWD2(false, false, false, false, 64), GS_BWD2(false, false, false, true, 64)},
              {GS_BWD2(false, false, true, false, 64), GS_BWD2(false, false, true, true, 64)}},
             {{GS_BWD2(false, true, false, false, 64), GS_BWD2(false, true, false, true, 64)},
              {GS_BWD2(false, true, true, false, 64), GS_BWD2(false, true, true, true, 64)}}},
            {{{GS_BWD2(true, false, false, false, 64), GS_BWD2(true, false, false, true, 64)},
              {GS_BWD2(true, false, true, false, 64), GS_BWD2(true, false, true, true, 64)}},
             {{GS_BWD2(true, true, false, false, 64), GS_BWD2(true, true, false, true, 64)},
              {GS_BWD2(true, true, true, false, 64), GS_BWD2(true, true, true, true, 64)}}}};
        return t[cull][atomic][persistent][any_c];
    }
    if (batch == 128 && cull) {
        static const RasterBwdKernel<float> t[2][2][2] = {
            {{GS_BWD2(true, false, false, false, 128), GS_BWD2(true, false, false, true, 128)},
             {GS_BWD2(true, false, true, false, 128), GS_BWD2(true, false, true, true, 128)}},
            {{GS_BWD2(true, true, false, false, 128), GS_BWD2(true, true, false, true, 128)},
             {GS_BWD2(true, true, true, false, 128), GS_BWD2(true, true, true, true, 128)}}};
        return t[atomic][persistent][any_c];
    }
#undef GS_BWD2
    return nullptr;
}

}  // namespace gs
