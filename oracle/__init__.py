"""Oracle for the Leuvenshtein hot path -- TEST INFRASTRUCTURE ONLY.

This package is the independent, slow, obviously-correct statement of what the
GPU library computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it; the
product library never does, and the two share no code.

Modules
-------
``plain``   plaintext algorithms: Wagner-Fischer (Eq. eq_wf), a breadth-first
            search over single edit operations (the definition of the edit
            distance in Section 2.3), the Myers cell equations (Section 2.3.3),
            the Leuvenshtein one-lookup cell (Eq. mye_eq_2, Eq. eq_keyeq2,
            Table LUTmin), the ASCII two-lookup equality (Algorithm alg_ascii),
            the preprocessing table (Section 5, Table tab_pre) and PBS counts
            (Table tab_pbs).
``tfhe``    the CPU TFHE restatement (``tfhe_oracle.c``: keygen, encryption,
            key switch, modulus switch, blind rotation with SCHOOLBOOK
            negacyclic products mod 2^64, sample extract) and the encrypted
            Leuvenshtein driver that follows Algorithm algo_complete.

Parity pins (see tests/test_oracle_*.py) tie every function to something other
than itself: worked examples printed in the paper (tests/golden/), brute force
on tiny inputs, closed forms and invariants.  The paper's own numeric TFHE
parameter set is not printed in the paper: ciphertext values for that set are
"parity unpinned"; the oracle is pinned for the parameter sets it is run with.
"""
