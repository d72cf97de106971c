// Register-tiled step kernels for R in {1, 2, 3, 4}.
#include "rows_step.cuh"

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

const TmaLauncher *tma_launcher_a(int R) {
    static const TmaLauncher m1 = make_tma_launcher<1>();
    static const TmaLauncher m2 = make_tma_launcher<2>();
    static const TmaLauncher m3 = make_tma_launcher<3>();
    static const TmaLauncher m4 = make_tma_launcher<4>();
    switch (R) {
        case 1: return &m1;
        case 2: return &m2;
        case 3: return &m3;
        case 4: return &m4;
        default: return nullptr;
    }
}

const RowsLauncher *rows_launcher_a(int R) {
    static const RowsLauncher w2 = make_rows_launcher<2>();
    static const RowsLauncher w4 = make_rows_launcher<4>();
    switch (R) {
        case 2: return &w2;
        case 4: return &w4;
        default: return nullptr;
    }
}

}  // namespace mfmc
