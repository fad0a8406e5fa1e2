"""FP64 CPU oracle for the P-SPIR PSF system matrix (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never does, and this package never imports the product path.

The arithmetic lives in ``psf_oracle.c`` (plain double-precision C, compiled
with gcc by :func:`build`); this module only marshals numpy arrays.  MLEM and
the Poisson log-likelihood, which are a few array expressions, are written
here on top of the C projectors.
"""
from .oracle import (  # noqa: F401
    build,
    lib_path,
    threads,
    sigma,
    node,
    gap_eq,
    face_point,
    trace_response,
    table_build,
    composed,
    spread,
    spread_topn,
    topn_bf16,
    sino_index,
    voxel_homog,
    lor_normal,
    tie_margin,
    tie_count,
    siddon,
    slabclip,
    rows_geom,
    window_pair,
    pair_row_map,
    rows_psf_dense,
    csr_fwd,
    csr_back,
    spread_apply,
    spread_adjoint,
    mlem,
    listmode_osem,
    poisson_loglik,
    poisson_grad,
    NORM_NONE,
    NORM_EFF,
    NORM_UNIT,
)
