// Register-tiled step kernels for R in {5, 6, 8}.
#include "rows_step.cuh"

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

const TmaLauncher *tma_launcher_b(int R) {
    static const TmaLauncher m5 = make_tma_launcher<5>();
    static const TmaLauncher m6 = make_tma_launcher<6>();
    static const TmaLauncher m8 = make_tma_launcher<8>();
    switch (R) {
        case 5: return &m5;
        case 6: return &m6;
        case 8: return &m8;
        default: return nullptr;
    }
}

const RowsLauncher *rows_launcher_b(int R) {
    static const RowsLauncher w6 = make_rows_launcher<6>();
    static const RowsLauncher w8 = make_rows_launcher<8>();
    switch (R) {
        case 6: return &w6;
        case 8: return &w8;
        default: return nullptr;
    }
}

}  // namespace mfmc
