// Register-tiled step kernels for R in {5, 6, 8}.
#include "step_kernels.cuh"

namespace mfmc {

const TileLauncher *tile_launcher_b(int R) {
    static const TileLauncher t5 = make_tile_launcher<5, true>();
    static const TileLauncher t6 = make_tile_launcher<6, true>();
    static const TileLauncher t8 = make_tile_launcher<8, true>();
    switch (R) {
        case 5: return &t5;
        case 6: return &t6;
        case 8: return &t8;
        default: return nullptr;
    }
}

}  // namespace mfmc
