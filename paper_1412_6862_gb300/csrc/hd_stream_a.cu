// hd_stream_a.cu -- compiled streaming-decoder configurations for n = 7, 15, 31
// (for n = 7 and 15 also with the decode table of hd_lut.cu).
#include "hd_stream.cuh"

namespace hd {

void register_stream_a(std::vector<StreamVariant> &v)
{
    // n = 7
    add_variants<7, 256, 4, 32, 0>(v);
    add_variants<7, 128, 4, 32, 1>(v);
    add_variants<7, 256, 3, 32, 1>(v);
    add_variants<7, 256, 4, 8, 1>(v);
    add_variants<7, 512, 2, 32, 1>(v);
    add_variants<7, 128, 4, 32, 1, false, true>(v);  // decode table
    add_variants<7, 512, 2, 32, 1, false, true>(v);
    // n = 15
    add_variants<15, 256, 4, 32, 0>(v);
    add_variants<15, 256, 4, 32, 1>(v);
    add_variants<15, 384, 3, 32, 1>(v);
    add_variants<15, 512, 2, 32, 1>(v);
    add_variants<15, 256, 4, 16, 1>(v);
    add_variants<15, 512, 2, 32, 1, false, true>(v);  // decode table (64 KB of shared memory per CTA)
    add_variants<15, 256, 2, 32, 1, false, true>(v);
    add_variants<15, 256, 3, 32, 1, false, true>(v);
    add_variants<15, 384, 2, 32, 1, false, true>(v);
    add_variants<15, 768, 2, 16, 1, false, true>(v);  // one CTA per SM: 24 warps beside the table
    add_variants<15, 640, 2, 32, 1, false, true>(v);
    add_variants<15, 576, 2, 32, 1, false, true>(v);  // 2^24 codewords: 6 chunks per warp
    add_variants<15, 576, 3, 32, 1, false, true>(v);
    add_variants<15, 512, 3, 32, 1, false, true>(v);
    add_variants<15, 512, 4, 32, 1, false, true>(v);
    add_variants<15, 640, 3, 32, 1, false, true>(v);
    add_variants<15, 512, 2, 32, 0, false, true>(v);  // separate output buffers: lookahead S
    add_variants<15, 576, 2, 32, 0, false, true>(v);
    add_variants<15, 640, 2, 32, 0, false, true>(v);
    add_variants<15, 576, 3, 32, 0, false, true>(v);
    add_variants<15, 1024, 2, 32, 1, false, true>(v);
    // n = 31
    add_variants<31, 128, 4, 32, 0>(v);
    add_variants<31, 128, 4, 32, 1>(v);
    add_variants<31, 128, 3, 32, 1>(v);
    add_variants<31, 256, 2, 32, 1>(v);
    add_variants<31, 256, 3, 16, 1>(v);
    add_variants<31, 96, 3, 32, 1>(v);
    add_variants<31, 96, 4, 32, 1>(v);
    add_variants<31, 64, 3, 32, 1>(v);
    add_variants<31, 128, 2, 32, 1>(v);  // 32 KB per CTA: 7 CTAs, 28 warps per SM
    add_variants<31, 64, 2, 32, 1>(v);
}

}  // namespace hd
