// wave_pass_r8.cu -- instantiations of the pass kernel for stencil radius 8 (SO 16).
#include "wave_pass.cuh"

namespace wave {

bool launch_pass_r8(int T, const CUtensorMap& mapA, const CUtensorMap& mapP, const CUtensorMap& mapK,
                    const PassArgs& a, int threads, size_t smem, long long blocks, cudaStream_t st, cudaError_t* err)
{
    switch (T) {
        case 1: *err = detail::launch_impl<8, 1>(mapA, mapP, mapK, a, threads, smem, blocks, st); return true;
        case 2: *err = detail::launch_impl<8, 2>(mapA, mapP, mapK, a, threads, smem, blocks, st); return true;
        default: return false;
    }
}

int pass_max_threads_r8(int T)
{
    switch (T) {
        case 1: return detail::Cfg<8, 1>::MAXT;
        case 2: return detail::Cfg<8, 2>::MAXT;
        default: return 0;
    }
}

int pass_prefetch_r8(int T)
{
    switch (T) {
        case 1: return detail::Cfg<8, 1>::D;
        case 2: return detail::Cfg<8, 2>::D;
        default: return 0;
    }
}

}  // namespace wave
