// rs_tag2.cu -- the tag strategy's kernels with two parents per lane and chunk (64-parent
// chunks, chosen when regions are short on average); the engine is in rs_tag.cuh.
#include "rs_tag.cuh"

namespace {
const TagEntry g_tag_kernels2[] = RS_TAG_TABLE(2);
}  // namespace

const TagEntry *rs_tag_table2(size_t *n)
{
    *n = sizeof g_tag_kernels2 / sizeof g_tag_kernels2[0];
    return g_tag_kernels2;
}
