// wave_pass_r8.cu -- instantiations of the pass kernel for stencil radius 8 (SO 16).
// Each entry is one (T, z quads per row, thread rows, queue storage) variant the
// autotuner can pick; queue storage 0/1 = registers (moved / rotated), 2 = tensor memory;
// variant 6 = warp-specialised pass with 2 rows per thread (tensor-memory queues).
#include "wave_lean.cuh"

namespace wave {

#define WAVE_SHAPE(T, QZ, RY, QM) \
    {8, T, QZ, RY, QM, detail::smem_bytes<8, T, QZ, RY>(), &detail::launch_impl<8, T, QZ, RY, QM>}
// variants 5 and 6: warp-specialised pass, NY = 1 or 2 rows per thread, x queues in tensor memory
#define WAVE_LEAN(T, QZ, RY, NY) \
    {8, T, QZ, RY, 4 + NY, detail::lean_smem_bytes<8, T, QZ, RY, NY>(), &detail::launch_lean<8, T, QZ, RY, NY>}

const PassShape* pass_shapes_r8(int* n)
{
    static const PassShape shapes[] = {
        WAVE_SHAPE(1, 16, 16, 0),
        WAVE_SHAPE(1, 8, 32, 0),
        WAVE_SHAPE(1, 16, 16, 1),
        WAVE_SHAPE(1, 16, 8, 2),
        WAVE_SHAPE(1, 16, 16, 2),
        WAVE_SHAPE(1, 16, 32, 2),
        WAVE_SHAPE(2, 8, 32, 0),
        WAVE_SHAPE(2, 8, 32, 1),
        WAVE_SHAPE(2, 8, 32, 2),
        WAVE_LEAN(1, 16, 32, 2),
        WAVE_LEAN(1, 8, 64, 2),
    };
    *n = static_cast<int>(sizeof(shapes) / sizeof(shapes[0]));
    return shapes;
}

}  // namespace wave
