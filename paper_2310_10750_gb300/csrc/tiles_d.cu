// Register-tiled step kernels for R in {16}.
#include "step_kernels.cuh"

namespace mfmc {

const TileLauncher *tile_launcher_d(int R) {
    static const TileLauncher t16 = make_tile_launcher<16, false>();
    switch (R) {
        case 16: return &t16;
        default: return nullptr;
    }
}

}  // namespace mfmc
