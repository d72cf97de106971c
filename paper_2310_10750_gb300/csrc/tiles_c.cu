// Register-tiled step kernels for R in {11, 12}.
#include "tma_step.cuh"

namespace mfmc {

const TileLauncher *tile_launcher_c(int R) {
    static const TileLauncher t11 = make_tile_launcher<11, false>();
    static const TileLauncher t12 = make_tile_launcher<12, false>();
    switch (R) {
        case 11: return &t11;
        case 12: return &t12;
        default: return nullptr;
    }
}

const TmaLauncher *tma_launcher_c(int R) {
    static const TmaLauncher m11 = make_tma_launcher<11>();
    static const TmaLauncher m12 = make_tma_launcher<12>();
    switch (R) {
        case 11: return &m11;
        case 12: return &m12;
        default: return nullptr;
    }
}

}  // namespace mfmc
