// Register-tiled step kernels for R in {16}.
#include "tma_step.cuh"

namespace mfmc {

const TileLauncher *tile_launcher_d(int R) {
    static const TileLauncher t16 = make_tile_launcher<16, false>();
    switch (R) {
        case 16: return &t16;
        default: return nullptr;
    }
}

const TmaLauncher *tma_launcher_d(int R) {
    static const TmaLauncher m16 = make_tma_launcher<16>();
    switch (R) {
        case 16: return &m16;
        default: return nullptr;
    }
}

}  // namespace mfmc
