// Register-tiled step kernels for R in {1, 2, 3, 4}.
#include "step_kernels.cuh"

namespace mfmc {

const TileLauncher *tile_launcher_a(int R) {
    static const TileLauncher t1 = make_tile_launcher<1, true>();
    static const TileLauncher t2 = make_tile_launcher<2, true>();
    static const TileLauncher t3 = make_tile_launcher<3, true>();
    static const TileLauncher t4 = make_tile_launcher<4, true>();
    switch (R) {
        case 1: return &t1;
        case 2: return &t2;
        case 3: return &t3;
        case 4: return &t4;
        default: return nullptr;
    }
}

}  // namespace mfmc
