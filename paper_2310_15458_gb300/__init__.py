"""GB300 (sm_103a) strong recursive skeletonization (RS-S).

The numerical work runs in ``librss_gb300.so`` (hand-written CUDA kernels
behind the C ABI of ``include/rss.h``); this package only marshals arguments.
Build the library with ``python -m paper_2310_15458_gb300.build``.  Loading
fails with an error if the library is missing: there is no CPU fallback.
"""
from .rss import (LAPLACE, HELMHOLTZ, TEST_POLY, TEST_RPOLY, HELMHOLTZ_LS, RSSError, Tree, Factor,
                  rss_build_tree, rss_factor, rss_solve, rss_solve_noalloc, rss_free, rss_info, rss_trim_memory,
                  rss_self_integral, rss_matvec, rss_solve_iterative, rss_probe_fp64, rss_probe_dmma, rss_tune_solve,
                  rss_level_ranks, rss_box_record, library_path,
                  Server, rss_server_create, rss_server_add, rss_server_submit,
                  rss_server_wait, rss_server_stats)

__all__ = ["LAPLACE", "HELMHOLTZ", "TEST_POLY", "TEST_RPOLY", "HELMHOLTZ_LS", "RSSError", "Tree", "Factor",
           "rss_build_tree", "rss_factor", "rss_solve", "rss_solve_noalloc", "rss_free", "rss_info", "rss_trim_memory",
           "rss_self_integral", "rss_matvec", "rss_solve_iterative", "rss_probe_fp64", "rss_probe_dmma", "rss_tune_solve",
           "rss_level_ranks", "rss_box_record", "library_path", "Server",
           "rss_server_create", "rss_server_add", "rss_server_submit", "rss_server_wait",
           "rss_server_stats"]
