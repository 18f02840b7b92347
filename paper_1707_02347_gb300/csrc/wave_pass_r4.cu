// wave_pass_r4.cu -- instantiations of the pass kernel for stencil radius 4 (SO 8).
#include "wave_pass.cuh"

namespace wave {

bool launch_pass_r4(int T, const CUtensorMap& mapA, const CUtensorMap& mapP, const CUtensorMap& mapK,
                    const PassArgs& a, int threads, size_t smem, long long blocks, cudaStream_t st, cudaError_t* err)
{
    switch (T) {
        case 1: *err = detail::launch_impl<4, 1>(mapA, mapP, mapK, a, threads, smem, blocks, st); return true;
        case 2: *err = detail::launch_impl<4, 2>(mapA, mapP, mapK, a, threads, smem, blocks, st); return true;
        case 3: *err = detail::launch_impl<4, 3>(mapA, mapP, mapK, a, threads, smem, blocks, st); return true;
        default: return false;
    }
}

int pass_max_threads_r4(int T)
{
    switch (T) {
        case 1: return detail::Cfg<4, 1>::MAXT;
        case 2: return detail::Cfg<4, 2>::MAXT;
        case 3: return detail::Cfg<4, 3>::MAXT;
        default: return 0;
    }
}

int pass_prefetch_r4(int T)
{
    switch (T) {
        case 1: return detail::Cfg<4, 1>::D;
        case 2: return detail::Cfg<4, 2>::D;
        case 3: return detail::Cfg<4, 3>::D;
        default: return 0;
    }
}

}  // namespace wave
