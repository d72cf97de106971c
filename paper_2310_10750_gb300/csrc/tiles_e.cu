// Register-tiled step kernels for R in {22, 24}.
#include "tma_step.cuh"

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

const TmaLauncher *tma_launcher_e(int R) {
    static const TmaLauncher m22 = make_tma_launcher<22>();
    static const TmaLauncher m24 = make_tma_launcher<24>();
    switch (R) {
        case 22: return &m22;
        case 24: return &m24;
        default: return nullptr;
    }
}

}  // namespace mfmc
