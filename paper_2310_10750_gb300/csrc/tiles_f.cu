// Register-tiled step kernels for R in {32}.
#include "tma_step.cuh"

namespace mfmc {

const TileLauncher *tile_launcher_f(int R) {
    static const TileLauncher t32 = make_tile_launcher<32, false>();
    switch (R) {
        case 32: return &t32;
        default: return nullptr;
    }
}

const TmaLauncher *tma_launcher_f(int R) {
    static const TmaLauncher m32 = make_tma_launcher<32>();
    switch (R) {
        case 32: return &m32;
        default: return nullptr;
    }
}

}  // namespace mfmc
