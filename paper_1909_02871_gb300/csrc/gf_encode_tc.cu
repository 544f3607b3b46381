// gf_encode_tc.cu -- bit-sliced GF(256) encode on tcgen05 tensor cores.
#include "gf_encode.h"
#include "gf_internal.cuh"

namespace gf {

bool bitsliced_available() { return false; }

long long bitsliced_tiles(const EncGen &, int &col_chunks, int &k_chunks)
{
    col_chunks = k_chunks = 0;
    return 0;
}

int launch_bitsliced(const EncodeBatch &, cudaStream_t) { return GF_ENOTSUP; }

}  // namespace gf
