// k_recip_long with traversal counting on (see pb_recip_long.cuh)
#include "pb_recip_long.cuh"

void launch_recip_long_counting(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots, uint32_t iter_base,
        int num_sms, cudaStream_t st) {
    k_recip_long<true><<<num_sms * 4, PH2_THREADS, 0, st>>>(S, T, P, B, slots, iter_base);
}
