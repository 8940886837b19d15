"""Plain CPU oracle of PAGANI's adaptive integration (test infrastructure).

ORACLE / TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
the cpu_baseline / --impl reference legs of bench.py may import anything from
here.  The product package (paper_2104_06494_gb300) never does, and the oracle
never imports the product: the two share no code.

* rule.py          the degree-9 rule and its four null rules, exact rationals
* closed_forms.py  closed-form integrals of the five synthetic families
* pagani_oracle.c  the algorithm step by step (Algorithms 2 and 3), plain C
* capi.py          ctypes front end and the gcc build of pagani_oracle.c
"""
