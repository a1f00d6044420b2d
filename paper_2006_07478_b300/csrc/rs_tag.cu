// rs_tag.cu -- the tag strategy's kernels with one parent per lane and chunk (32-parent
// chunks), and the choice among all tag kernels.  The engine is in rs_tag.cuh; the
// two-parents-per-lane kernels are compiled separately in rs_tag2.cu.
#include "rs_tag.cuh"

namespace {
const TagEntry g_tag_kernels1[] = RS_TAG_TABLE(1);
}  // namespace

// the specialised kernel of P's stage list for P.V and P.cpl, else the generic one
const void *rs_tag_kernel_entry(const KParams &P)
{
    int ops[5] = {0, 0, 0, 0, 0};
    ops[0] = (int)P.st[0].op;
    for (int i = 1; i < P.n_stages - 1 && i < 5; ++i) ops[i] = (int)P.st[i].op;
    size_t n = sizeof g_tag_kernels1 / sizeof g_tag_kernels1[0];
    const TagEntry *t = P.cpl == 2 ? rs_tag_table2(&n) : g_tag_kernels1;
    const void *generic = nullptr;
    for (size_t k = 0; k < n; ++k) {
        const TagEntry &e = t[k];
        if (e.V != (int)P.V) continue;
        if (e.oe == 0) {
            generic = e.fn;
            continue;
        }
        // a specialised kernel ends in the sink it was compiled for
        if ((e.emit != 0) == (P.emit != 0) && e.oe == ops[0] && e.o1 == ops[1] && e.o2 == ops[2] &&
            e.o3 == ops[3] && e.o4 == ops[4])
            return e.fn;
    }
    return generic;
}

int rs_tag_kernel_is_specialised(const KParams &P)
{
    const void *f = rs_tag_kernel_entry(P);
    size_t n = sizeof g_tag_kernels1 / sizeof g_tag_kernels1[0];
    const TagEntry *t = P.cpl == 2 ? rs_tag_table2(&n) : g_tag_kernels1;
    for (size_t k = 0; k < n; ++k)
        if (t[k].fn == f) return t[k].oe != 0;
    return 0;
}
