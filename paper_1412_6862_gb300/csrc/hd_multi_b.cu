// hd_multi_b.cu -- compiled multi-packet streaming configurations for n = 63,
// 127 and 255: the single-stream decoder's built-in chunk geometry per n.
#include "hd_multi.cuh"

namespace hd {

void register_multi_b(std::vector<MultiVariant> &v)
{
    add_multi_variants<63, 64, 2, 32, 1>(v);
    add_multi_variants<127, 256, 3, 8, 1>(v);
    add_multi_variants<255, 128, 2, 8, 1>(v);
}

}  // namespace hd
