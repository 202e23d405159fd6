// Tensor-core (tcgen05) SpMVs on the brick/tile layout.
#include "life_internal.cuh"

namespace life {

life_status build_tile_layout(life_index_s* ix, cudaStream_t s) {
    (void)ix; (void)s;
    set_error("tensor-core layout not available in this build");
    return LIFE_ENOTSUP;
}

life_status dsc_tc(life_index_s*, const float*, const float*, const float*, float*, double*, int*,
                   const life_sbb_state*, int, cudaStream_t) {
    set_error("tensor-core DSC not available in this build");
    return LIFE_ENOTSUP;
}

life_status wc_tc(life_index_s*, const float*, const float*, float*, const life_sbb_state*, int, cudaStream_t) {
    set_error("tensor-core WC not available in this build");
    return LIFE_ENOTSUP;
}

}  // namespace life
