// Sorting of 64-bit keys (the Step-2 block keys) with CUB's device radix sort.
#include <cub/device/device_radix_sort.cuh>

#include "mra_internal.cuh"

namespace mra {

// keys[0..n) sorted ascending in place (stream-ordered)
int sort_keys_u64(const Alloc& A, uint64_t* keys, int n, cudaStream_t st) {
    if (n <= 1) return MRA_OK;
    Scratch tmpmem(A);
    uint64_t* out;
    MRA_TRY(tmpmem.get(&out, (size_t)n));
    size_t tmp_bytes = 0;
    MRA_CK(cub::DeviceRadixSort::SortKeys(nullptr, tmp_bytes, (const unsigned long long*)keys,
                                          (unsigned long long*)out, n, 0, 64, st));
    unsigned char* tmp;
    MRA_TRY(tmpmem.get(&tmp, tmp_bytes));
    MRA_CK(cub::DeviceRadixSort::SortKeys(tmp, tmp_bytes, (const unsigned long long*)keys, (unsigned long long*)out,
                                          n, 0, 64, st));
    MRA_CK(cudaMemcpyAsync(keys, out, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    return MRA_OK;
}

}  // namespace mra
