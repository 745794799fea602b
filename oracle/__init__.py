"""CPU FP64 oracle for the FDP=H space-time BIEM hot path (Sato & Ando, arXiv 1903.02118).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the package
``paper_1903_02118_gb300`` and its CUDA library) may import, call or link
anything here.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle is written from the paper alone, in plain numpy FP64, and shares no
code, tables or constants with the CUDA path.  Modules:

* ``kernel``  -- the discrete 2-D antiplane kernel K_{i,j,m} (Sec. 2.1.2,
  Eq. 4; closed form re-derived from the 2-D SH Green's function, since the
  paper only cites it) and its static limit.
* ``dense``   -- the plain ST-BIEM time march T_n = sum_m K_m D_{n-m}
  (Eq. 4), the "original" method of the paper.
* ``fdph``    -- the FDP=H plan built by the paper's rules (bounding-box
  clustering, Eqs. 8-9 admissibility, ART integers of Eq. 30 and App. C.3,
  amplitude terms Eq. 28, waveforms Eq. 29, Domain S of App. B.1, 2-D
  transient of App. B.3 / App. H, dense inadmissible leaves of App. E) and the
  brute-force evaluation of the compressed operator it defines.

Parity status of each function is stated in its module header.
"""
