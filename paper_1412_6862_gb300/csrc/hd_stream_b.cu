// hd_stream_b.cu -- compiled streaming-decoder configurations for n = 63.
#include "hd_stream.cuh"

namespace hd {

void register_stream_b(std::vector<StreamVariant> &v)
{
    add_variants<63, 128, 3, 32, 1>(v);
    add_variants<63, 128, 2, 32, 1>(v);
    add_variants<63, 192, 2, 32, 1>(v);
    add_variants<63, 256, 3, 16, 1>(v);
    add_variants<63, 128, 4, 16, 1>(v);
    add_variants<63, 128, 3, 32, 0>(v);
    add_variants<63, 64, 2, 32, 1>(v);  // 32 KB per CTA: 7 CTAs, 14 warps per SM
    add_variants<63, 64, 3, 32, 1>(v);
}

}  // namespace hd
