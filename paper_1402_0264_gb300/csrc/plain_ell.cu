// The block-size study of the plain product (polymul_plain_ell): the CTA
// kernel of plain.cu instantiated with 4 and 16 warps per block (l = 128 and
// 512 threads), in a translation unit of its own so that both compile in
// parallel.  plain.cu's non-template kernels, launchers and entry points are
// left out here (PM_PLAIN_STUDY_TU); its templates are shared.
#define PM_PLAIN_STUDY_TU
#include "plain.cu"
