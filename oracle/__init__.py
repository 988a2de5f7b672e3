"""The oracle: a plain, slow FP64 CPU statement of the method of Serov &
Sergeeva, arXiv:1505.06707 (ECS + split-operator FFT, Sec. II; PCG with the
FFT preconditioners, Sec. III).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
GPU library (``paper_1505_06707_gb300``) and never imports it.
"""
