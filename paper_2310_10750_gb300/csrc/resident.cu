// Resident (whole field in shared memory) kernels for R in {1, ..., 6, 8}.
#include "rows_step.cuh"

namespace mfmc {

ResidentFn resident_launcher(int R) {
    switch (R) {
        case 1: return &launch_resident<1>;
        case 2: return &launch_resident<2>;
        case 3: return &launch_resident<3>;
        case 4: return &launch_resident<4>;
        case 5: return &launch_resident<5>;
        case 6: return &launch_resident<6>;
        case 8: return &launch_resident<8>;
        default: return nullptr;
    }
}

const TileLauncher *tile_launcher_a(int R);
const TileLauncher *tile_launcher_b(int R);
const TileLauncher *tile_launcher_c(int R);
const TileLauncher *tile_launcher_d(int R);
const TileLauncher *tile_launcher_e(int R);
const TileLauncher *tile_launcher_f(int R);

const TmaLauncher *tma_launcher_a(int R);
const TmaLauncher *tma_launcher_b(int R);
const TmaLauncher *tma_launcher_c(int R);
const TmaLauncher *tma_launcher_d(int R);
const TmaLauncher *tma_launcher_e(int R);
const TmaLauncher *tma_launcher_f(int R);

const TmaLauncher *tma_launcher(int R) {
    const TmaLauncher *(*groups[6])(int) = {tma_launcher_a, tma_launcher_b, tma_launcher_c,
                                            tma_launcher_d, tma_launcher_e, tma_launcher_f};
    for (auto g : groups)
        if (const TmaLauncher *t = g(R)) return t;
    return nullptr;
}

const RowsLauncher *rows_launcher_a(int R);
const RowsLauncher *rows_launcher_b(int R);

const RowsLauncher *rows_launcher(int R) {
    if (const RowsLauncher *r = rows_launcher_a(R)) return r;
    return rows_launcher_b(R);
}

const TileLauncher *tile_launcher(int R) {
    const TileLauncher *(*groups[6])(int) = {tile_launcher_a, tile_launcher_b, tile_launcher_c,
                                             tile_launcher_d, tile_launcher_e, tile_launcher_f};
    for (auto g : groups)
        if (const TileLauncher *t = g(R)) return t;
    return nullptr;
}

}  // namespace mfmc
