// hd_stream_a.cu -- compiled streaming-decoder configurations for n = 7, 15, 31.
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
    // n = 15
    add_variants<15, 256, 4, 32, 0>(v);
    add_variants<15, 256, 4, 32, 1>(v);
    add_variants<15, 384, 3, 32, 1>(v);
    add_variants<15, 512, 2, 32, 1>(v);
    add_variants<15, 256, 4, 16, 1>(v);
    // n = 31
    add_variants<31, 128, 4, 32, 0>(v);
    add_variants<31, 128, 4, 32, 1>(v);
    add_variants<31, 128, 3, 32, 1>(v);
    add_variants<31, 256, 2, 32, 1>(v);
    add_variants<31, 256, 3, 16, 1>(v);
}

}  // namespace hd
