// Register-tiled step kernels for R in {22, 24}.
#include "step_kernels.cuh"

namespace mfmc {

const TileLauncher *tile_launcher_e(int R) {
    static const TileLauncher t22 = make_tile_launcher<22, false>();
    static const TileLauncher t24 = make_tile_launcher<24, false>();
    switch (R) {
        case 22: return &t22;
        case 24: return &t24;
        default: return nullptr;
    }
}

}  // namespace mfmc
