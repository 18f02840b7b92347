// wave_pass_r2.cu -- instantiations of the pass kernel for stencil radius 2 (SO 4).
// Each entry is one (T, z quads per row, thread rows, queue storage) variant the
// autotuner can pick; queue storage 0/1 = registers (moved / rotated), 2 = tensor memory;
// variant 4 = two-step pass with skewed wavefront tiling in y (tensor-memory queues);
// variants 5, 6 = warp-specialised pass with 1 or 2 rows per thread (tensor-memory queues).
#include "wave_lean.cuh"
#include "wave_skew.cuh"

namespace wave {

#define WAVE_SHAPE(T, QZ, RY, QM) \
    {2, T, QZ, RY, QM, detail::smem_bytes<2, T, QZ, RY>(), &detail::launch_impl<2, T, QZ, RY, QM>}
// variants 5 and 6: warp-specialised pass, NY = 1 or 2 rows per thread, x queues in tensor memory
#define WAVE_LEAN(T, QZ, RY, NY) \
    {2, T, QZ, RY, 4 + NY, detail::lean_smem_bytes<2, T, QZ, RY, NY>(), &detail::launch_lean<2, T, QZ, RY, NY>}
// variant 7: warp-specialised pass, 2 rows per thread, x queues as tensor-memory shift registers
#define WAVE_LEAN7(T, QZ, RY) \
    {2, T, QZ, RY, 7, detail::lean_smem_bytes<2, T, QZ, RY, 2, true>(), &detail::launch_lean<2, T, QZ, RY, 2, true>}
// variant 4: skewed wavefront tiling in y, T = 2, x queues in tensor memory
#define WAVE_SKEW(QZ, RY) {2, 2, QZ, RY, 4, detail::skew_smem_bytes<2, QZ, RY>(), &detail::launch_skew<2, QZ, RY>}

const PassShape* pass_shapes_r2(int* n)
{
    static const PassShape shapes[] = {
        WAVE_SHAPE(1, 16, 16, 0),
        WAVE_SHAPE(1, 32, 8, 0),
        WAVE_SHAPE(1, 8, 32, 0),
        WAVE_SHAPE(1, 16, 16, 1),
        WAVE_SHAPE(1, 16, 16, 2),
        WAVE_SHAPE(1, 16, 8, 2),
        WAVE_SHAPE(1, 16, 32, 2),
        WAVE_SHAPE(2, 16, 16, 0),
        WAVE_SHAPE(2, 8, 32, 0),
        WAVE_SHAPE(2, 16, 24, 0),
        WAVE_SHAPE(2, 16, 16, 1),
        WAVE_SHAPE(2, 16, 24, 2),
        WAVE_SHAPE(2, 16, 32, 2),
        WAVE_SHAPE(2, 8, 64, 2),
        WAVE_SHAPE(3, 8, 32, 0),
        WAVE_SHAPE(3, 16, 24, 0),
        WAVE_SHAPE(3, 8, 32, 1),
        WAVE_SHAPE(3, 16, 24, 2),
        WAVE_SHAPE(3, 16, 32, 2),
        WAVE_SHAPE(4, 8, 32, 0),
        WAVE_SHAPE(4, 16, 24, 0),
        WAVE_SHAPE(4, 8, 32, 1),
        WAVE_SHAPE(4, 8, 32, 2),
        WAVE_SKEW(16, 32),
        WAVE_LEAN(2, 16, 32, 1),
        WAVE_LEAN(2, 16, 40, 1),
        WAVE_LEAN(2, 16, 44, 1),
        WAVE_LEAN(3, 16, 32, 1),
        WAVE_LEAN(1, 16, 8, 1),
        WAVE_LEAN(1, 16, 16, 1),
        WAVE_LEAN7(2, 16, 44),
        WAVE_LEAN7(3, 16, 44),
    };
    *n = static_cast<int>(sizeof(shapes) / sizeof(shapes[0]));
    return shapes;
}

}  // namespace wave
