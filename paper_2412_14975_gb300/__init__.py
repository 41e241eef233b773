"""GB300 RID recognizer: Python binding of the C ABI in ``include/ridfa.h`` (libridfa.so).

Argument marshalling only: every step of recognition runs in the library's sm_103a kernels.
The binding loads ``libridfa.so`` from this directory and raises ImportError when it is missing
(build it with ``python paper_2412_14975_gb300/build_lib.py``); there is no fallback.

Device buffers may be given as CUDA tensors (anything with ``data_ptr()``) or as raw integer
addresses; ``stream`` may be a ``torch.cuda.Stream``, a raw ``cudaStream_t`` integer, or None
(the current torch stream when torch is imported, else the legacy default stream).
"""

from ._lib import (RIDFA_MAX_SLOTS, RIDFA_MAX_STATES, RIDFA_NOALLOC_SCRATCH_BYTES,  # noqa: F401
                   RIDFA_UNDEF, Program, RidfaError, ridfa_recognize_noalloc,
                   ridfa_bench_hbm_read, ridfa_bench_smem_gather,
                   Tuning, lib_path, ridfa_compile, ridfa_delegates, ridfa_export_tables,
                   ridfa_free, ridfa_last_plan, ridfa_last_status, ridfa_last_timings, ridfa_program_info, ridfa_recognize,
                   ridfa_recognize_async, ridfa_recognize_dfa, ridfa_recognize_dfa_async, ridfa_recognize_nfa, ridfa_recognize_host, ridfa_check_bounded_wait,
                   ridfa_slots, ridfa_state_set, ridfa_strerror,
                   Batch, ridfa_batch_create, ridfa_batch_run, ridfa_batch_get_stats, ridfa_batch_free,
                   ridfa_recognize_batch, Server, RIDFA_SUBMIT_DEVICE_TEXT, ridfa_count_transitions, ridfa_cpu_recognize,
                   ShardSummary, ridfa_recognize_shard, ridfa_join_shards, ridfa_join_scan)
